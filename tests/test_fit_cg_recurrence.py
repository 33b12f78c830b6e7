"""The fitting CG as the GPU arranges it, restated in FP64 on the CPU and held
against the oracle's CG (Sec. 4.1).

The GPU forms each direction before the residual that defines its beta exists,
so beta's numerator r.r(it + 1) comes from the recurrence
rr - 2 alpha r.q + alpha^2 q.q over the sums of the same pass, while alpha
takes the norm of the stored residual.  In exact arithmetic the two CG forms
are the same iteration; these tests show they agree to rounding on fitting
systems, and that the arrangement stops moving once an iterate is exact (the
case where taking alpha from the recurrence as well breaks down)."""
import numpy as np
import pytest

from oracle import Fitting, Tomography
from synth import configs


def cg_beta_recurrence(A, b, a0, iters, alpha_from_recurrence=False, rr0_ulps=0):
    """CG with beta = rr_next / rr, rr_next = rr - 2 alpha r.q + alpha^2 q.q;
    alpha = r.r / p.q with r.r of the stored residual (or, with
    alpha_from_recurrence, the recurrence's value carried over, starting from
    the initial r.r moved by rr0_ulps units in the last place, as a sum taken
    in another order may be)."""
    a = np.array(a0, dtype=np.float64, copy=True)
    r = b - A(a)
    p = r.copy()
    rr_carried = float(r @ r)
    for _ in range(rr0_ulps):
        rr_carried = float(np.nextafter(rr_carried, np.inf))
    for _ in range(iters):
        q = A(p)
        pq, rq, qq = float(p @ q), float(r @ q), float(q @ q)
        rr = rr_carried if alpha_from_recurrence else float(r @ r)
        if pq == 0.0 and rr == 0.0:
            alpha = 0.0
        else:
            alpha = rr / pq
        rr_next = max(0.0, rr - 2.0 * alpha * rq + alpha * alpha * qq)
        beta = rr_next / rr if rr != 0.0 else 0.0
        a = a + alpha * p
        r = r - alpha * q
        p = r + beta * p
        rr_carried = rr_next
    return a


def _small():
    g = configs.small_lgs_config(16, 32, 3, 2)
    return configs.with_fitting(g, altitudes=(0.0, 4000.0, 9000.0), pitches=(0.5, 0.72, 1.0),
                                field_arcmin=1.2, n_dir=3)


def _single():
    g = configs.small_lgs_config(16, 32, 3, 2)
    return configs.with_fitting(g, altitudes=(0.0,), pitches=(0.5,), field_arcmin=0.0, n_dir=1)


@pytest.mark.parametrize("warm", [False, True])
def test_recurrence_beta_matches_the_oracle_cg(warm):
    g = _small()
    fit, tom = Fitting(g), Tomography(g)
    rng = np.random.default_rng(41)
    b = fit.rhs(tom.synthesis(rng.standard_normal(tom.n)))
    a0 = 0.1 * rng.standard_normal(fit.n) if warm else np.zeros(fit.n)
    for iters in (1, 2, 4, 8):
        want = fit.cg(b, a0, iters)
        got = cg_beta_recurrence(fit.apply_normal, b, a0, iters)
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), iters


def test_exact_iterate_stays_put_only_with_the_stored_norm():
    """One mirror on the sampling points seen from one direction: H^T H is the
    identity on the reached actuators and CG is exact after one iteration."""
    g = _single()
    fit, tom = Fitting(g), Tomography(g)
    d = fit.apply_normal_diagonal()
    assert set(np.unique(d)) <= {0.0, 1.0}
    b = fit.rhs(tom.synthesis(np.random.default_rng(42).standard_normal(tom.n)))
    for iters in (1, 2, 12):
        got = cg_beta_recurrence(fit.apply_normal, b, np.zeros(fit.n), iters)
        assert np.array_equal(got, fit.cg(b, np.zeros(fit.n), iters))
        assert np.allclose(got, b, rtol=0, atol=1e-12 * np.abs(b).max())
    # stored norms: a first r.r summed in another order changes nothing
    got = cg_beta_recurrence(fit.apply_normal, b, np.zeros(fit.n), 12, rr0_ulps=1)
    assert np.allclose(got, b, rtol=0, atol=1e-12 * np.abs(b).max())
    # alpha from the recurrence as well: that one unit in the last place leaves
    # a residue where r.r is zero, and alpha = residue / p.q throws the iterate off
    with np.errstate(all="ignore"):
        bad = cg_beta_recurrence(fit.apply_normal, b, np.zeros(fit.n), 12, alpha_from_recurrence=True,
                                 rr0_ulps=1)
        assert not np.all(np.isfinite(bad)) or np.linalg.norm(bad - b) > np.linalg.norm(b)
