"""CPU checks of the C-ABI library: it builds, loads, exports every symbol that
include/sci.h declares, and rejects bad arguments before touching the GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sci.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sci_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2005_08028_gb300 import build as b
    path = b.build()
    import paper_2005_08028_gb300.sci as s
    return s.load(path)


def test_header_declares_expected_calls():
    names = declared_functions()
    for must in ("sci_forward", "sci_adjoint", "sci_project", "sci_tv_prox", "sci_gap_tv",
                 "sci_admm_tv", "sci_masks_pack"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_version(lib):
    assert lib.sci_version() >= 10000
    for code in range(7):
        assert lib.sci_status_str(code)


def test_argument_errors_return_before_any_launch(lib):
    from paper_2005_08028_gb300.sci import SciParams
    fake = C.c_void_p(0x10000)  # never dereferenced: validation fails first
    prm = SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1)
    # null y
    assert lib.sci_gap_tv(None, fake, 8, 8, 2, C.byref(prm), fake, fake, None, 0, fake, 1 << 30, None) == 1
    # B > 32
    assert lib.sci_gap_tv(fake, fake, 8, 8, 33, C.byref(prm), fake, fake, None, 0, fake, 1 << 30, None) == 2
    # non-positive sizes
    assert lib.sci_forward(fake, fake, 0, 8, 2, fake, None) == 1
    # lambda <= 0 and non-finite lambda
    bad = SciParams(0, -1.0, 0.0, 10, 5, 0, 0, 1, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(bad), fake, fake, None, 0, fake, 1 << 30, None) == 1
    nan = SciParams(0, float("nan"), 0.0, 10, 5, 0, 0, 1, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(nan), fake, fake, None, 0, fake, 1 << 30, None) == 4
    # S = 0, bad TV type, negative rho for ADMM
    s0 = SciParams(0, 0.05, 0.0, 10, 0, 0, 0, 1, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(s0), fake, fake, None, 0, fake, 1 << 30, None) == 1
    tv9 = SciParams(9, 0.05, 0.0, 10, 5, 0, 0, 1, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(tv9), fake, fake, None, 0, fake, 1 << 30, None) == 1
    dual7 = SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 7)  # neither FGP (0), Chambolle (1) nor Clip (2)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(dual7), fake, fake, None, 0, fake, 1 << 30, None) == 1
    clip_itv = SciParams(1, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 2)  # the Clip box is an ATV solver
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(clip_itv), fake, fake, None, 0, fake, 1 << 30, None) == 1
    assert lib.sci_tv_prox_clip(fake, 8, 8, 2, 2, 0.05, 5, C.c_void_p(0x20000), fake, 1 << 30, None) == 1
    assert lib.sci_tv_prox_cham(fake, 8, 8, 2, 0, 0.05, 5, fake, fake, 1 << 30, None) == 1  # x aliases theta
    neg = SciParams(0, 0.05, -0.5, 10, 5, 0, 0, 1, 1)
    assert lib.sci_admm_tv(fake, fake, 8, 8, 2, C.byref(neg), fake, fake, fake, None, 0, fake, 1 << 30,
                           None) == 1
    # workspace too small / misaligned
    need = lib.sci_solver_workspace(8, 8, 2, C.byref(prm))
    assert need > 0
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(prm), fake, fake, None, 0, fake, need - 1, None) == 6
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(prm), fake, fake, None, 0, C.c_void_p(0x10010),
                          need, None) == 6
    # resid_every without a buffer
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(prm), fake, fake, None, 3, fake, need, None) == 1
    # prox: aliasing and bad inner_iters
    assert lib.sci_tv_prox(fake, 8, 8, 2, 0, 0.05, 5, fake, fake, 1 << 30, None) == 1
    assert lib.sci_tv_prox(fake, 8, 8, 2, 0, 0.05, 0, C.c_void_p(0x20000), fake, 1 << 30, None) == 1
    # projection: negative rho, x aliasing theta
    assert lib.sci_project(fake, None, fake, fake, 8, 8, 2, -1.0, C.c_void_p(0x20000), None) == 1
    assert lib.sci_project(fake, None, fake, fake, 8, 8, 2, 0.0, fake, None) == 1


def test_warm_start_arguments(lib):
    """The dual warm start: 0 or 1; GAP and ADMM on the temporally blocked
    path only (not FISTA, not fuse_k = -1, not VTV with B > 24); it needs
    room for two pairs of carried dual fields in the workspace."""
    from paper_2005_08028_gb300.sci import SciParams
    fake = C.c_void_p(0x10000)  # never dereferenced: validation fails first
    big = 1 << 40
    cold = SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0)
    warm = SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 1)
    two = SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 2)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(two), fake, fake, None, 0, fake, big, None) == 1
    per_update = SciParams(0, 0.05, 0.0, 10, 5, 0, -1, 1, 1, 0, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(per_update), fake, fake, None, 0, fake, big, None) == 1
    assert lib.sci_fista_tv(fake, fake, 8, 8, 2, C.byref(warm), fake, fake, None, 0, fake, big, None) == 1
    vtv32 = SciParams(2, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 1)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 32, C.byref(vtv32), fake, fake, None, 0, fake, big, None) == 1
    N, es = 64 * 48 * 4, 4
    grow = lib.sci_solver_workspace(64, 48, 4, C.byref(warm)) - lib.sci_solver_workspace(64, 48, 4, C.byref(cold))
    assert grow >= 4 * N * es
    need = lib.sci_solver_workspace(64, 48, 4, C.byref(warm))
    assert lib.sci_admm_tv(fake, fake, 64, 48, 4, C.byref(warm), fake, fake, fake, None, 0, fake, need - 1,
                           None) == 6


def test_workspace_sizes_scale(lib):
    from paper_2005_08028_gb300.sci import SciParams
    p32 = SciParams(0, 0.05, 0.01, 10, 5, 0, 0, 1, 1)
    p16 = SciParams(0, 0.05, 0.01, 10, 5, 1, 0, 1, 1)
    a = lib.sci_solver_workspace(512, 512, 10, C.byref(p32))
    b = lib.sci_solver_workspace(512, 512, 10, C.byref(p16))
    N = 512 * 512 * 10
    assert a >= 7 * N * 4  # xt + three 2-field dual buffers
    assert b >= 9 * N * 2  # plus theta and u copies in 16-bit
    assert lib.sci_tv_prox_workspace(64, 64, 4, 0) >= 6 * 64 * 64 * 4 * 4


def _header_struct_fields(name):
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    body = re.search(r"typedef struct \{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        parts = [p.strip() for p in decl.split(",")]
        ctype, first = parts[0].rsplit(None, 1)
        ctype = ctype.replace(" ", "")
        for name in [first] + parts[1:]:  # declarators sharing one base type
            stars = len(name) - len(name.lstrip("*"))
            fields.append((ctype + "*" * stars, name.lstrip("*")))
    return fields


@pytest.mark.parametrize("cname,pyname", [("sci_params", "SciParams"), ("sci_problem", "SciProblem")])
def test_binding_structs_mirror_the_header(cname, pyname):
    """The ctypes mirrors of the ABI structs have the header's fields, in its
    order, with matching widths (the binding renames lambda to lam only)."""
    import paper_2005_08028_gb300.sci as s
    width = {"int": C.c_int, "float": C.c_float}
    header = _header_struct_fields(cname)
    mirror = getattr(s, pyname)._fields_
    assert len(header) == len(mirror)
    for (ctype, cfield), (pfield, ptype) in zip(header, mirror):
        assert pfield == {"lambda": "lam"}.get(cfield, cfield)
        if ctype in width:
            assert ptype is width[ctype], (cfield, ctype, ptype)
        else:  # pointers
            assert C.sizeof(ptype) == C.sizeof(C.c_void_p), (cfield, ctype)


def test_fuse_depth_planner(lib):
    """Host logic, no GPU: dual updates per temporally blocked launch.  One-frame
    tiles (ATV, ITV2D) take up to 10; the 32 x 32 VTV tiles of up to 10 frames
    take up to 6 by default (and at most 7: halo <= 8); 16 / 24 frames take up
    to 3 (halo <= 4); more than 24 frames fall back to one launch per update
    (0).  fuse_k = -1 switches blocking off; fuse_k > 0 caps the depth; S caps
    it too."""
    import paper_2005_08028_gb300.sci as s
    q = s.sci_fused_updates
    assert q("atv", 10, 10) == 10 and q("itv2d", 32, 10) == 10
    assert q("atv", 10, 25) == 10 and q("atv", 10, 4) == 4
    assert q("vtv", 10, 10) == 6 and q("vtv", 8, 10) == 6 and q("vtv", 10, 5) == 5
    assert q("vtv", 16, 10) == 3 and q("vtv", 24, 5) == 3
    assert q("vtv", 25, 10) == 0 and q("vtv", 32, 10) == 0
    assert q("atv", 10, 10, -1) == 0 and q("vtv", 10, 10, -1) == 0
    assert q("atv", 10, 10, 3) == 3 and q("vtv", 10, 10, 30) == 7  # clamped to the halo


def _problems(sizes, ptr=0x10000):
    import paper_2005_08028_gb300.sci as s
    arr = (s.SciProblem * max(1, len(sizes)))()
    for k, (nx, ny, B) in enumerate(sizes):
        arr[k] = s.SciProblem(nx, ny, B, ptr, ptr, ptr, None)  # pointers are never dereferenced here
    return arr


def test_batched_workspace_planner(lib):
    """Host logic, no GPU: the batched solver's workspace holds, per
    measurement, two pixel fields (R^+, r) and eleven storage-type voxel
    fields (x-tilde, two theta, eight carried duals), each 256-byte aligned,
    behind a descriptor table; invalid batches report 0."""
    import paper_2005_08028_gb300.sci as s

    def ws(sizes, tv=2, storage=0, lam=0.05, fuse_k=0):
        prm = s.SciParams(tv, lam, 0.0, 10, 5, storage, fuse_k, 1, 1, 0)
        return lib.sci_gap_tv_batched_workspace(_problems(sizes), len(sizes), C.byref(prm))

    def al(b):
        return (b + 255) // 256 * 256

    def fields(sizes, es):
        return sum(2 * al(nx * ny * 4) + 11 * al(nx * ny * B * es) for nx, ny, B in sizes)

    mix = [(128, 128, 8), (256, 256, 8), (37, 70, 10), (48, 40, 24)]
    for storage, es in ((0, 4), (1, 2), (2, 2)):
        w = ws(mix, storage=storage)
        table = w - fields(mix, es)
        assert 0 < table <= al(1024 * len(mix)) and table % 256 == 0, (storage, table)
    assert ws(mix, storage=2) < ws(mix, storage=0)
    # the table grows with the count, the fields with the sizes; depth does not matter
    assert ws(mix + [(16, 16, 8)]) > ws(mix)
    assert ws(mix, fuse_k=2) == ws(mix) == ws(mix, fuse_k=-1)
    # one-frame TV forms take any B up to 32; VTV only up to 24
    assert ws([(64, 64, 32)], tv=0) > 0 and ws([(64, 64, 32)], tv=1) > 0
    assert ws([(64, 64, 25)], tv=2) == 0
    assert ws([(64, 64, 33)], tv=0) == 0
    # invalid arguments
    assert ws([]) == 0
    assert ws(mix, lam=0.0) == 0 and ws(mix, lam=float("nan")) == 0
    assert ws([(0, 16, 8)]) == 0 and ws([(16, 16, 0)]) == 0
    assert ws(mix, storage=3) == 0 and ws(mix, fuse_k=-2) == 0
    prm = s.SciParams(2, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0)
    assert lib.sci_gap_tv_batched_workspace(_problems([(16, 16, 8)], ptr=None), 1, C.byref(prm)) == 0
    assert lib.sci_gap_tv_batched_workspace(_problems(mix), len(mix), None) == 0


def test_fault_injection_on_the_host(lib):
    """Failures made on the host, before any launch (no GPU needed): an empty
    batch, one bad descriptor in an otherwise valid mixed batch (a null
    measurement, B > 32, VTV with B > 24), options the batched driver does not
    run, and check_input outside {0, 1}.  Each call returns its status
    without touching the (never dereferenced) device pointers."""
    import paper_2005_08028_gb300.sci as s
    fake = C.c_void_p(0x10000)
    mix = [(128, 128, 8), (256, 256, 8), (37, 70, 10), (48, 40, 24)]
    prm = s.SciParams(2, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0, 0)
    big = 1 << 40
    assert lib.sci_gap_tv_batched(_problems([]), 0, C.byref(prm), fake, big, None) == 1  # empty batch
    assert lib.sci_gap_tv_batched_workspace(_problems([]), 0, C.byref(prm)) == 0
    probs = _problems(mix)
    probs[2].y = None  # one measurement without data
    assert lib.sci_gap_tv_batched(probs, len(mix), C.byref(prm), fake, big, None) == 1
    probs = _problems(mix)
    probs[1].B = 40  # more frames than a mask word holds
    assert lib.sci_gap_tv_batched(probs, len(mix), C.byref(prm), fake, big, None) == 2
    probs = _problems(mix)
    probs[3].B = 30  # VTV tiles hold at most 24 frames
    assert lib.sci_gap_tv_batched(probs, len(mix), C.byref(prm), fake, big, None) == 2
    for fields in ((2, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 1, 0),   # warm start
                   (2, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0, 1),   # check_input
                   (0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 2, 0, 0)):  # Clip box
        bad = s.SciParams(*fields)
        assert lib.sci_gap_tv_batched(_problems(mix), len(mix), C.byref(bad), fake, big, None) == 1, fields
    chk2 = s.SciParams(0, 0.05, 0.0, 10, 5, 0, 0, 1, 1, 0, 0, 2)
    assert lib.sci_gap_tv(fake, fake, 8, 8, 2, C.byref(chk2), fake, fake, None, 0, fake, big, None) == 1
