"""The library's FRAP time-scale fit (``sbg_frap_fit``, Sec. 3.3) is host
code: checked here without a GPU against curves whose scale is known
exactly, against the oracle's fit on the same curves, and on its argument
checks."""
import numpy as np
import pytest

import oracle
from paper_2304_11165_b300 import SbgError
from paper_2304_11165_b300 import _abi
from paper_2304_11165_b300.api import frap_fit


def test_exact_scale_on_the_reference_grid():
    t = np.linspace(0, 10, 41)
    tr = np.linspace(0, 10, 4001)
    s, rss = frap_fit(t, 1 - np.exp(-0.37 * t), tr, 1 - np.exp(-tr), 0.01, 1.0)
    assert abs(s - 0.37) <= 1e-12 and rss <= 1e-24


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_matches_the_oracle_fit(seed):
    rng = np.random.default_rng(seed)
    true_s = rng.uniform(0.2, 0.9)
    t = np.linspace(0, 8, 33)
    tr = np.linspace(0, 8, 257)
    f = 1 - np.exp(-true_s * t) * (1 + 0.1 * np.sin(t)) + rng.normal(0, 1e-3, t.size)
    g = 1 - np.exp(-tr) * (1 + 0.1 * np.sin(tr / true_s))
    s, rss = frap_fit(t, f, tr, g, 0.05, 1.0)
    so, rsso = oracle.frap_fit(t, f, tr, g, 0.05, 1.0)
    # the minimiser of a smooth residual is fixed to about sqrt(machine epsilon)
    # relative, its value to machine precision
    assert abs(s - so) <= 1e-7 and abs(rss - rsso) <= 1e-10 * rsso


def test_argument_checks():
    t = np.linspace(0, 1, 5)
    with pytest.raises(SbgError) as e:
        frap_fit(t, t, t[::-1].copy(), t, 0.1, 1.0)   # reference times decrease
    assert e.value.status == _abi.SBG_ERR_INVALID_ARG
    with pytest.raises(SbgError):
        frap_fit(t, t, t, t, 0.1, 2.0)                # reference shorter than s_hi * t_max
    with pytest.raises(SbgError):
        frap_fit(t, t, t, t, 0.0, 1.0)                # s_lo must be positive
    with pytest.raises(SbgError):
        frap_fit(t, np.full(5, np.nan), t, t, 0.1, 1.0)


def test_effective_D_and_tau_from_the_fit():
    """sbg_frap_effective_D (Eq. 2): a bulk reference recorded at D_ref = 0.7
    fitted with the exact scale 0.37 gives D_eff = 0.37 * 0.7 and tau = 1/0.37;
    a measured curve equal to the reference gives D_eff = D_ref, tau = 1."""
    from paper_2304_11165_b300.api import frap_effective_D
    t = np.linspace(0, 10, 41)
    tr = np.linspace(0, 10, 4001)
    d_eff, tau, s, rss = frap_effective_D(t, 1 - np.exp(-0.37 * t), tr, 1 - np.exp(-tr), 0.7, 0.01, 1.0)
    assert abs(s - 0.37) <= 1e-12 and abs(d_eff - 0.37 * 0.7) <= 1e-12 and abs(tau - 1 / 0.37) <= 1e-11
    assert rss <= 1e-24
    d1, tau1, s1, _ = frap_effective_D(tr, 1 - np.exp(-tr), tr, 1 - np.exp(-tr), 0.7, 0.01, 1.0)
    assert abs(s1 - 1.0) <= 1e-12 and abs(d1 - 0.7) <= 1e-12 and abs(tau1 - 1.0) <= 1e-12
    with pytest.raises(SbgError):
        frap_effective_D(t, t, tr, tr, 0.0, 0.01, 1.0)    # D_ref must be positive
