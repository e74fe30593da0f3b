"""Sussman redistancing on the GPU (Sec. 2.1) against the FP64 oracle at the
same iteration count, its invariants (sign preservation, phi = 0 fixed), the
host and device entry paths, early stopping, and the level set feeding the
sparse-grid build on the device."""
import numpy as np
import pytest

import oracle
from workloads import grf_geometry

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2304_11165_b300 import Grid, SbgError, redistance  # noqa: E402
from paper_2304_11165_b300 import _abi  # noqa: E402


def blob_indicator(shape, seed):
    rng = np.random.default_rng(seed)
    f = rng.normal(size=shape)
    for _ in range(3):  # a little smoothing so that the phases form blobs
        f = (f + np.roll(f, 1, 0) + np.roll(f, 1, 1) + np.roll(f, 1, 2)) / 4
    return np.where(f > 0, 1.0, -1.0)


def ball(n):
    h = 4.0 / n
    c = -2.0 + (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    return np.where(r < 1.0, 1.0, -1.0), 1.0 - r, h


@pytest.mark.parametrize("shape,dx", [((17, 19, 23), (1.0, 0.9, 1.1)), ((9, 40, 33), (0.5, 0.5, 0.5)),
                                      ((1, 21, 37), (1.0, 1.0, 1.0))])
def test_fp64_matches_the_oracle(shape, dx):
    phi0 = blob_indicator(shape, 3)
    ref = oracle.sussman(phi0, dx=dx, cfl=0.3, iters=45)
    out, it, _ = redistance(phi0, dx=dx, cfl=0.3, max_iter=45)
    assert it == 45
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_fp32_matches_the_oracle_on_the_unit_ball():
    ind, sdf, h = ball(64)
    ref = oracle.sussman(ind, dx=(h, h, h), cfl=0.3, iters=60)
    out, _, _ = redistance(ind.astype(np.float32), dx=(h, h, h), cfl=0.3, max_iter=60)
    assert out.dtype == np.float32
    assert np.max(np.abs(out - ref)) <= 2e-6 * np.max(np.abs(ref))
    band = np.abs(sdf) < 2 * h
    assert np.max(np.abs(out[band] - sdf[band])) <= 0.35 * h


def test_sign_and_zero_are_preserved():
    phi0 = blob_indicator((20, 24, 28), 4).astype(np.float32)
    phi0[5, 6, 7] = 0.0
    out, _, _ = redistance(phi0, cfl=0.33, max_iter=80)
    assert np.all(np.sign(out) == np.sign(phi0))
    assert out[5, 6, 7] == 0.0


def test_device_path_equals_host_path_and_in_place_allowed():
    phi0 = blob_indicator((24, 20, 30), 5).astype(np.float32)
    host, _, _ = redistance(phi0, max_iter=37)
    d = torch.from_numpy(phi0).cuda()
    dev, it, _ = redistance(d, max_iter=37)
    assert isinstance(dev, torch.Tensor) and dev.is_cuda and it == 37
    np.testing.assert_array_equal(host, dev.cpu().numpy())


def test_early_stop_matches_the_oracle_at_the_same_count():
    ind, _, h = ball(40)
    out, it, res = redistance(ind, dx=(h, h, h), cfl=0.3, max_iter=2000, tol=1e-3, band=2.0, check_every=8)
    assert it < 2000 and it % 8 == 0 and res < 1e-3
    ref = oracle.sussman(ind, dx=(h, h, h), cfl=0.3, iters=it)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_redistanced_indicator_builds_the_same_pore_space():
    phi_true = grf_geometry(64, 77, 0.45, ell=4.0)
    ind = torch.from_numpy(np.where(phi_true > 0, 1.0, -1.0).astype(np.float32)).cuda()
    phi, _, _ = redistance(ind, max_iter=120)
    g = Grid(phi, block=4)
    host = phi.cpu().numpy()
    eps = np.finfo(np.float32).eps
    assert g.n_active == int((host > eps).sum())
    assert np.all(np.sign(host) == ind.cpu().numpy())
    # features thinner than two voxels keep their sign but shrink towards 0
    # (why the paper filters them out of the indicator first); they are few here
    n_pore = int((phi_true > eps).sum())
    assert n_pore - g.n_active <= 1e-3 * n_pore
    assert g.info["n_band_blocks"] > 0


def test_argument_checks():
    phi0 = np.ones((4, 4, 4))
    with pytest.raises(SbgError) as e:
        redistance(phi0, cfl=0.4)   # 0.4 * 3 > 1 for isotropic spacing
    assert e.value.status == _abi.SBG_ERR_INVALID_ARG
    with pytest.raises(SbgError):
        redistance(phi0, dx=(1.0, 0.0, 1.0))
    with pytest.raises(SbgError):
        redistance(phi0, check_every=0)
    out, it, res = redistance(phi0, max_iter=0)
    assert it == 0 and np.isnan(res)
    np.testing.assert_array_equal(out, phi0)
