"""The decoders' phi(x) = ln(1 + 2/(e^x - 1)) against FP64 over the range the
sum-product decoders use, [phi(20), 20]: the library-function form within a few
binary32 ulps, the fast forms (hardware approximations plus Taylor series where
a difference cancels; in nats for the adjoint, in bits for the layered and
flooding check node) within 3e-5 relative."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def phi64(x):
    return np.log1p(2.0 / np.expm1(x))


@pytest.fixture(scope="module")
def lx():
    import paper_2203_11854_gb300 as lx
    assert torch.cuda.is_available()
    lx.load_library()
    return lx


def grid():
    lo = phi64(20.0)
    x = np.concatenate([np.geomspace(lo, 20.0, 400001), np.linspace(0.05, 0.08, 20001),  # series switch
                        np.array([lo, 0.0625, np.nextafter(np.float32(0.0625), np.float32(0)), 20.0])])
    return np.unique(x.astype(np.float32))


@pytest.mark.parametrize("fast,bound", [(0, 2e-6), (1, 3e-5), (2, 3e-5)])
def test_phi_relative_error(lx, fast, bound):
    x = grid()
    got = lx.ldpcx_phi(torch.from_numpy(x).cuda(), fast=fast).cpu().numpy().astype(np.float64)
    ref = phi64(x.astype(np.float64))
    rel = np.abs(got - ref) / ref
    assert np.isfinite(got).all()
    assert rel.max() <= bound, f"max relative error {rel.max():.3g} at x = {x[rel.argmax()]!r}"


@pytest.mark.parametrize("fast", [1, 2])
def test_phi_is_decreasing_involution(lx, fast):
    # phi(phi(x)) = x, and phi decreases; checks the fast forms' two branches join
    x = grid()
    y = lx.ldpcx_phi(torch.from_numpy(x).cuda(), fast=fast)
    yy = lx.ldpcx_phi(y.clamp(min=float(x[0]), max=20.0).contiguous(), fast=fast).cpu().numpy()
    mid = (x > 1e-3) & (x < 15.0)
    assert np.allclose(yy[mid], x[mid], rtol=1e-3)
    yc = y.cpu().numpy().astype(np.float64)
    assert (np.diff(yc) <= 3e-5 * yc[1:]).all()  # non-increasing up to the stated error
