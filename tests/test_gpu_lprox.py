"""Learned prox on the GPU against the FP64 network oracle.

The tensor-core convolution is compared with the oracle on the same
BF16-rounded operands; the whole network's output and gradients are compared
within BF16 tolerances (activations are stored in BF16 between layers); a
few Adam steps must lower the loss; the kernels' bounded waits never fire.
"""
import numpy as np
import pytest

from oracle import lprox_oracle as L
from gpu_helpers import lib, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    return lib()


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


@pytest.mark.parametrize("shape", [(1, 2, 3, 64), (2, 3, 5, 70), (1, 4, 2, 200), (3, 1, 1, 1)])
@pytest.mark.parametrize("relu", [False, True])
def test_tensor_core_conv_matches_oracle(pkg, shape, relu):
    n, D, H, W = shape
    rng = np.random.default_rng(sum(shape) + relu)
    act = bf16_round(rng.normal(size=(n, D, H, W, 32)))
    w = bf16_round(rng.normal(size=(27, 32, 32)) * 0.1)
    b = rng.normal(size=32).astype(np.float32)
    dev = torch.device("cuda")
    out, err = pkg.sci_conv3d_c32_bf16(torch.from_numpy(act).to(dev).to(torch.bfloat16).contiguous(),
                                       torch.from_numpy(w).to(dev).to(torch.bfloat16).contiguous(),
                                       torch.from_numpy(b).to(dev), relu=relu)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    got = out.float().cpu().numpy()
    for k in range(n):
        ref = L.conv3d(act[k], w, b if relu else np.zeros(32))
        if relu:
            ref = np.maximum(ref, 0.0)
        # FP32 accumulation of exact BF16 products; output rounded to BF16
        np.testing.assert_allclose(got[k], ref, rtol=8e-3, atol=1e-3 * float(np.abs(ref).max() + 1))


def _params(seed, C=32):
    ps = L.init_params(C=C, seed=seed)
    ps[3] = (ps[3][0] * 10.0, ps[3][1])  # make f visible
    flat = np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in ps]).astype(np.float32)
    return ps, flat


def test_network_forward_matches_oracle(pkg):
    ps, flat = _params(7)
    rng = np.random.default_rng(8)
    x = rng.random((2, 4, 12, 70)).astype(np.float32)
    net = pkg.LearnedProx(params=torch.from_numpy(flat).cuda())
    th = net.apply(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    assert net.error_word((2, 4, 12, 70), False) == 0
    for k in range(2):
        ref, _ = L.lprox_forward(x[k], ps)
        f_ref = ref - x[k]
        f_got = th[k].cpu().numpy() - x[k]
        rms = float(np.sqrt(np.mean(f_ref ** 2)))
        assert np.abs(f_got - f_ref).max() <= 0.05 * rms + 1e-4, (np.abs(f_got - f_ref).max(), rms)


# rows of 20 voxels (one padded tile of the tensor-core weight gradient) and
# of 70 (three tiles, the last one partly padding), frames and rows that put
# every (dz, dy) tap over the volume's edges
@pytest.mark.parametrize("shape", [(2, 3, 10, 20), (1, 4, 5, 70)])
def test_network_gradients_match_oracle(pkg, shape):
    ps, flat = _params(9)
    rng = np.random.default_rng(10)
    x = rng.random(shape).astype(np.float32)
    t = (x + 0.05 * rng.normal(size=x.shape)).astype(np.float32)
    net = pkg.LearnedProx(params=torch.from_numpy(flat).cuda())
    g, loss = net.grads(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    g = g.cpu().numpy().astype(np.float64)
    # the oracle's mean is over all voxels of every volume
    tot = None
    nv = x.shape[0]
    for k in range(nv):
        lk, gk = L.lprox_loss_and_grads(x[k], t[k], ps)
        flat_k = np.concatenate([np.concatenate([dw.reshape(-1), db]) for dw, db in gk])
        tot = flat_k / nv if tot is None else tot + flat_k / nv
    # per layer: direction and size; per tap (27) and per output channel: the
    # slice's relative error, so a wrong tap or channel is located; per entry:
    # no gradient entry off by more than a tenth of the layer's largest.  The
    # bounds allow for BF16 weights and activations (8-bit mantissa) with FP32
    # accumulation against the FP64 oracle.
    shapes = [(27, 32, 1), (32,), (27, 32, 32), (32,), (27, 32, 32), (32,), (27, 1, 32), (1,)]
    off = 0
    for shp in shapes:
        sz = int(np.prod(shp))
        a, b = g[off:off + sz], tot[off:off + sz]
        off += sz
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert cos > 0.995 and abs(np.linalg.norm(a) / np.linalg.norm(b) - 1) < 0.03, (shp, cos)
        assert np.abs(a - b).max() <= 0.1 * np.abs(b).max(), shp
        if len(shp) == 3:
            # a slice's error against its own size, but not below a floor of
            # 5% of the layer's largest slice: BF16 operands put a noise floor
            # proportional to the layer's scale under slices that are nearly
            # zero (an output channel whose ReLU is rarely open), while a wrong
            # tap or channel errs by the order of its own slice
            A, Bm = a.reshape(shp), b.reshape(shp)
            tap_n = [np.linalg.norm(Bm[tap]) for tap in range(27)]
            for tap in range(27):
                d = np.linalg.norm(A[tap] - Bm[tap]) / max(tap_n[tap], 0.05 * max(tap_n), 1e-30)
                assert d < 0.1, (shp, "tap", tap, d)
            out_n = [np.linalg.norm(Bm[:, o]) for o in range(shp[1])]
            for o in range(shp[1]):
                d = np.linalg.norm(A[:, o] - Bm[:, o]) / max(out_n[o], 0.05 * max(out_n), 1e-30)
                assert d < 0.1, (shp, "out", o, d)


def test_training_lowers_loss(pkg):
    rng = np.random.default_rng(11)
    x = rng.random((4, 4, 16, 64)).astype(np.float32)
    t = (0.5 * x + 0.25).astype(np.float32)
    _, flat = _params(12)
    net = pkg.LearnedProx(params=torch.from_numpy(flat).cuda())
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    losses = [float(net.train_step(xd, td, 1e-3).item()) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0]
    assert net.error_word(x.shape, True) == 0
