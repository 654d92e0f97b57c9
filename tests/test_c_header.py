"""CPU: include/sci.h is a plain C interface.  A C99 program (and the same
source as C++17) compiled with warnings as errors includes it, links
libsci.so and calls entry points that need no GPU: the version, every
status string, the fuse-depth planner and argument rejection.  The struct
sizes it prints must equal the Python binding's mirrors."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "sci.h"

int main(void) {
    int k, bad = 0;
    sci_params p;
    int cands[2] = {5, -1};
    float ms[2];
    int best = 7;
    memset(&p, 0, sizeof p);
    p.tv = SCI_TV_VTV;
    p.lambda = 0.05f;
    p.outer_iters = 10;
    p.inner_iters = 10;
    p.storage = SCI_F32;
    p.init = 1;
    for (k = SCI_OK; k <= SCI_ERR_WORKSPACE; ++k)
        if (sci_status_str((sci_status)k) == NULL || sci_status_str((sci_status)k)[0] == 0) bad = 1;
    /* argument errors return before anything touches a GPU */
    if (sci_tune_fuse(SCI_ALGO_GAP, NULL, NULL, 8, 8, 2, &p, NULL, NULL, NULL, 0, cands, 0, 1, 1, ms, &best,
                      NULL) != SCI_ERR_ARG) bad = 1;
    if (sci_gap_tv(NULL, NULL, 8, 8, 2, &p, NULL, NULL, NULL, 0, NULL, 0, NULL) != SCI_ERR_ARG) bad = 1;
    printf("version %d\n", sci_version());
    printf("fused %d %d %d\n", sci_fused_updates(SCI_TV_ATV, 1, 10, 0), sci_fused_updates(SCI_TV_VTV, 10, 10, 0),
           sci_fused_updates(SCI_TV_VTV, 32, 10, 0));
    printf("sizes %u %u\n", (unsigned)sizeof(sci_params), (unsigned)sizeof(sci_problem));
    printf("best %d bad %d\n", best, bad);
    return bad;
}
"""


def _compile_and_run(tmp_path, compiler, flags, lib_dir):
    src = tmp_path / ("prog.c" if "gcc" in compiler else "prog.cpp")
    src.write_text(PROGRAM)
    exe = tmp_path / ("prog_" + os.path.basename(compiler).replace("+", "p"))
    cmd = [compiler, *flags, "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
           "-L", lib_dir, "-lsci", f"-Wl,-rpath,{lib_dir}", "-o", str(exe)]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    return dict(line.split(" ", 1) for line in out.stdout.strip().splitlines())


@pytest.fixture(scope="module")
def lib_dir():
    from paper_2005_08028_gb300 import build as b
    return os.path.dirname(b.build())


@pytest.mark.parametrize("compiler,flags", [("gcc", ["-std=c99", "-pedantic"]), ("g++", ["-std=c++17", "-pedantic"])])
def test_header_compiles_links_and_answers_without_a_gpu(tmp_path, lib_dir, compiler, flags):
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not found")
    from paper_2005_08028_gb300 import sci as S
    out = _compile_and_run(tmp_path, compiler, flags, lib_dir)
    lib = S.load()
    assert int(out["version"]) == lib.sci_version()
    assert out["fused"].split() == [str(S.sci_fused_updates("atv", 1, 10)), str(S.sci_fused_updates("vtv", 10, 10)),
                                    "0"]
    assert out["sizes"].split() == [str(C.sizeof(S.SciParams)), str(C.sizeof(S.SciProblem))]
    assert out["best"] == "7 bad 0"  # *best untouched on an argument error
