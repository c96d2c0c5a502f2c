"""Failure paths of the C ABI, made on the host (no GPU fault, no hang).

- A bounded wait of the tensor-core TTM that runs out (its limit shortened to one
  cycle with CP_OPT_WAIT_LIMIT): the kernel drains its copies in flight, frees its
  tensor memory and returns; the next synchronising call reports CP_ETIMEOUT, the
  context is poisoned (CP_ESTATE afterwards) and a new context on the same GPU
  works normally.
- Normal equations that are singular even after the shift (two all-zero factors
  make every Gamma(n) the zero matrix): CP_ENOTSPD, and the context stays usable.
- A NaN entry in a factor: CP_ENUMERIC from the sweep and from cp_fit.
"""
import numpy as np
import pytest

import synth
from oracle import cp_oracle as co

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CP_ENOTSPD, CP_ENUMERIC, CP_ETIMEOUT, CP_ESTATE = 4, 5, 6, 7


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__ as ge
    ge.build()
    import paper_2010_12056_gb300 as p
    return p


def problem(dims, R, seed):
    T64, _, A0 = synth.make_problem(seed, dims, R, eta=1e-2)
    T32 = np.ascontiguousarray(T64.astype(np.float32))
    return torch.from_numpy(T32).cuda(), T32.astype(np.float64), A0


def relerr(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["f16x3", "tf32x3"])
def test_wait_that_runs_out_reports_timeout(pkg, prec):
    dims, R = (128, 96, 140), 64
    Td, Tref, A0 = problem(dims, R, 91)
    ctx = pkg.CPContext(Td, R, A0=A0, prec=prec)
    ctx.set_option("wait_limit", 1)          # every wait that is not met at once runs out
    with pytest.raises(pkg.CPError) as e:
        ctx.sweep_dt(1)
    assert e.value.code == CP_ETIMEOUT
    assert "bounded device wait" in str(e.value)
    with pytest.raises(pkg.CPError) as e2:   # poisoned from now on
        ctx.sweep_msdt(1)
    assert e2.value.code == CP_ESTATE
    ctx.close()
    # the GPU and a new context are unaffected
    ok = pkg.CPContext(Td, R, A0=A0, prec=prec)
    for n in range(3):
        assert relerr(ok.mttkrp(n).cpu().numpy(), co.mttkrp(Tref, A0, n)) <= 1e-5
    assert ok.stats()["ttm_tensor_core"] >= 1
    ok.close()


def test_wait_limit_option_validated(pkg):
    Td, _, A0 = problem((16, 12, 20), 4, 92)
    ctx = pkg.CPContext(Td, 4, A0=A0, prec="f16x3")
    with pytest.raises(pkg.CPError) as e:
        ctx.set_option("wait_limit", -1)
    assert e.value.code == 1
    ctx.set_option("wait_limit", 0)          # back to the default
    ctx.sweep_dt(1)
    ctx.close()


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_singular_normal_equations_report_notspd(pkg, prec):
    dims, R = (40, 36, 44), 6
    Td, Tref, A0 = problem(dims, R, 93)
    ctx = pkg.CPContext(Td, R, A0=A0, prec=prec)
    ctx.set_factor(0, np.zeros_like(A0[0]))
    ctx.set_factor(1, np.zeros_like(A0[1]))  # every Gamma(n) has a zero Gram factor
    with pytest.raises(pkg.CPError) as e:
        ctx.sweep_dt(1)
    assert e.value.code == CP_ENOTSPD
    # not poisoned: new factors, and the sweeps follow the oracle from there
    for n in range(3):
        ctx.set_factor(n, A0[n])
    ctx.sweep_dt(3)
    ref = co.cp_als(Tref, A0, 3, route="dt")
    _, r = ctx.fit(exact=True)
    assert abs(r - co.residual_direct(Tref, ref.A)) <= 1e-6
    ctx.close()


def test_nan_factor_reports_enumeric(pkg):
    """The NaN is put in the last factor: the first update of a sweep does not read
    its own factor, so a NaN in factor 0 would be overwritten by finite values."""
    dims, R = (40, 36, 44), 6
    Td, _, A0 = problem(dims, R, 94)
    ctx = pkg.CPContext(Td, R, A0=A0, prec="f16x3")
    bad = A0[2].copy()
    bad[3, 2] = np.nan
    ctx.set_factor(2, bad)
    with pytest.raises(pkg.CPError) as e:
        ctx.fit(exact=True)
    assert e.value.code == CP_ENUMERIC
    with pytest.raises(pkg.CPError) as e:
        ctx.sweep_msdt(1)
    assert e.value.code == CP_ENUMERIC
    ctx.close()
