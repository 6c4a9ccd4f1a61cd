"""Dense NNLS by Algorithm 1 on the GPU (the paper's efficiency experiment)
against the FP64 oracle: aligned and ragged shapes, several right-hand sides,
a warm start from a given iterate and accumulator, host and device pointers."""
import numpy as np
import pytest

from oracle.dense_nnls import spgd_dense
from paper_1901_09266_gb300 import dode
from tests.helpers import rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


def _instance(nr, nc, m, seed):
    rng = np.random.default_rng(seed)
    B = (rng.standard_normal((nr, nc)) / np.sqrt(nc)).astype(np.float32)
    x = np.abs(rng.standard_normal((nc, m))) * (rng.random((nc, m)) < 0.7)
    Y = (B.astype(np.float64) @ x + 0.01 * rng.standard_normal((nr, m))).astype(np.float32)
    return B, Y


@pytest.mark.parametrize("nr,nc,m", [(512, 512, 1), (300, 257, 3), (1000, 64, 8), (33, 700, 2)])
def test_dense_spgd_matches_oracle(nr, nc, m):
    B, Y = _instance(nr, nc, m, seed=nr + nc + m)
    X, G, loss, ms = dode.dense_nnls(B, Y, 60, 0.05)
    Xo, Go, lo = spgd_dense(B, Y, 60, 0.05)
    # loss: 1e-5 relative, with a floor at FP32 resolution of the problem's scale
    # (1e-8 of ||y||^2) for underdetermined cases whose loss goes to ~0
    floor = 1e-8 * (Y.astype(np.float64) ** 2).sum(axis=0)
    np.testing.assert_allclose(loss, lo, rtol=1e-5, atol=floor.max())
    assert rel_norm(X, Xo, axis=0).max() < 1e-4
    assert np.all(X >= 0) and ms > 0
    # continuing from the returned state equals a longer run
    X2, G2, loss2, _ = dode.dense_nnls(B, Y, 40, 0.05, X0=X, G0=G)
    Xo2, _, lo2 = spgd_dense(B, Y, 100, 0.05)
    np.testing.assert_allclose(loss2, lo2, rtol=1e-5, atol=floor.max())
    assert rel_norm(X2, Xo2, axis=0).max() < 1e-4


def test_dense_spgd_device_pointers_and_errors():
    torch = pytest.importorskip("torch")
    B, Y = _instance(256, 256, 2, seed=5)
    Xh, _, lh, _ = dode.dense_nnls(B, Y, 30, 0.05)
    Bd, Yd = torch.from_numpy(B).cuda(), torch.from_numpy(Y).cuda()
    Xd, Gd, ld, _ = dode.dense_nnls(Bd, Yd, 30, 0.05)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Xd.cpu().numpy(), Xh)
    np.testing.assert_array_equal(ld.cpu().numpy(), lh)
    with pytest.raises(dode.DodeError) as e:
        dode.dense_nnls(B, np.zeros((256, 9), np.float32), 1, 0.05)      # more than 8 right-hand sides
    assert e.value.code == dode.ERR_ARG


@pytest.mark.parametrize("nr,nc", [(512, 512), (1003, 1024), (130, 8192), (2000, 4), (301, 6000), (77, 2048)])
def test_dense_one_pass_matches_two_passes_and_oracle(nr, nc):
    """One pass over B per iteration (rows staged by bulk asynchronous copies)
    against the two-pass kernels and the FP64 oracle; ragged row blocks and
    the largest supported column count included."""
    B, Y = _instance(nr, nc, 1, seed=nr * 7 + nc)
    X1, G1, l1, _ = dode.dense_nnls(B, Y, 40, 0.05, method=1)
    X2, G2, l2, _ = dode.dense_nnls(B, Y, 40, 0.05, method=2)
    Xo, _, lo = spgd_dense(B, Y, 40, 0.05)
    floor = 1e-8 * float((Y.astype(np.float64) ** 2).sum())
    np.testing.assert_allclose(l1, lo, rtol=1e-5, atol=floor)
    np.testing.assert_allclose(l2, lo, rtol=1e-5, atol=floor)
    assert rel_norm(X1, Xo, axis=0).max() < 1e-4
    assert rel_norm(X1, X2, axis=0).max() < 1e-5
    # one pass does not apply to several right-hand sides
    with pytest.raises(dode.DodeError) as e:
        dode.dense_nnls(B, np.concatenate([Y, Y], axis=1), 1, 0.05, method=1)
    assert e.value.code == dode.ERR_UNSUPPORTED


def test_dense_one_pass_wait_runs_out_then_recovers():
    """Failure path of the one-pass kernel without a GPU fault: with a wait limit
    of 0 polls every bounded wait for a row copy gives up at once, the call
    returns DODE_ERR_DEVICE_TIMEOUT after the kernel let its copies in flight
    land, and the next call in the same process matches the oracle."""
    B, Y = _instance(1003, 1024, 1, seed=9)
    dode.dense_set_wait_limit(0)
    try:
        with pytest.raises(dode.DodeError) as e:
            dode.dense_nnls(B, Y, 5, 0.05, method=1)
        assert e.value.code == dode.ERR_DEVICE_TIMEOUT
    finally:
        dode.dense_set_wait_limit(1 << 26)
    X, _, loss, _ = dode.dense_nnls(B, Y, 20, 0.05, method=1)
    Xo, _, lo = spgd_dense(B, Y, 20, 0.05)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(X, Xo, axis=0).max() < 1e-4
    with pytest.raises(dode.DodeError):
        dode.dense_set_wait_limit(-1)


@pytest.mark.parametrize("nr,nc,m", [(512, 512, 16), (1000, 764, 64), (260, 1024, 256), (300, 640, 128), (4, 36, 32)])
def test_dense_tensor_cores_match_tf32_oracle(nr, nc, m):
    """Many right-hand sides stacked into GEMMs on the tensor cores (method 3:
    tcgen05 with TF32 operands and FP32 accumulation).  Against the oracle's
    TF32 definition (the same operands, FP64 products and sums) the only
    differences are FP32 accumulation and rounding, which can move an operand's
    cut to TF32 by one TF32 unit (2^-10 relative) on a few elements: 1e-3
    normwise on X and on the loss.  Against the FP64 oracle the TF32 operands
    (relative error below 2^-10 each) move X by 4e-4 to 5e-4 normwise after 30
    steps on the square and tall instances and by 1.2e-2 on the wide one (260
    rows, 1024 columns: underdetermined, so the iterates are less constrained);
    the bound is 2e-2.  Ragged M and K tiles (1000 rows, 764 columns) and the
    largest tile (m = 256) included."""
    from oracle.dense_nnls import spgd_dense_tf32
    B, Y = _instance(nr, nc, m, seed=nr + 3 * nc + m)
    X, G, loss, ms = dode.dense_nnls(B, Y, 30, 0.05, method=3)
    Xt, _, lt = spgd_dense_tf32(B, Y, 30, 0.05)
    Xo, _, lo = spgd_dense(B, Y, 30, 0.05)
    e_t = rel_norm(X, Xt, axis=0).max()
    e_o = rel_norm(X, Xo, axis=0).max()
    print(f"tensor cores {nr}x{nc}, m={m}: X vs TF32 oracle {e_t:.2e}, vs FP64 oracle {e_o:.2e}, "
          f"loss vs TF32 {np.max(np.abs(loss - lt) / lt):.2e}")
    assert e_t < 1e-3
    np.testing.assert_allclose(loss, lt, rtol=1e-3)
    assert e_o < 2e-2
    assert np.all(X >= 0) and ms > 0


def test_dense_tensor_cores_device_pointers_and_limits():
    torch = pytest.importorskip("torch")
    B, Y = _instance(384, 512, 32, seed=17)
    Xh, Gh, lh, _ = dode.dense_nnls(B, Y, 10, 0.05, method=3)
    Bd, Yd = torch.from_numpy(B).cuda(), torch.from_numpy(Y).cuda()
    Xd, Gd, ld, _ = dode.dense_nnls(Bd, Yd, 10, 0.05, method=3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(Xd.cpu().numpy(), Xh)
    np.testing.assert_array_equal(ld.cpu().numpy(), lh)
    # continuing from the returned state equals a longer run
    X2, _, l2, _ = dode.dense_nnls(B, Y, 10, 0.05, X0=Xh, G0=Gh, method=3)
    X20, _, l20, _ = dode.dense_nnls(B, Y, 20, 0.05, method=3)
    np.testing.assert_array_equal(X2, X20)
    for bad_m in (8, 24):                                         # m must be a multiple of 16
        with pytest.raises(dode.DodeError) as e:
            dode.dense_nnls(B, np.zeros((384, bad_m), np.float32), 1, 0.05, method=3)
        assert e.value.code == dode.ERR_UNSUPPORTED
