"""The maximum-time-step protocol of the speed-up runs (largest stable fine
step with M = 1, then the largest M whose coarse step M dt_f is stable),
on the small test sphere, and for interfaces of one and of three cells."""
import pytest

from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import maxdt
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphw():
    return W.workload("scvt_2562")


@pytest.mark.parametrize("layers", [1, 3])
def test_max_dt_protocol(sphw, layers):
    w = sphw
    T = 30 * w.dt
    res = maxdt.max_dt_protocol(w.mesh, w.fine_mask, w.h0, w.u0, w.g, w.dt / w.M, T, M_max=12,
                                layers=layers)
    # the fine step is at least the CFL-0.5 step the workload was built with
    # (its fine CFL is 0.44), and LTS allows M of at least the resolution ratio
    assert res["dt_fine"] >= 0.9 * w.dt / w.M
    assert res["M_max_stable"] >= 2
    # the answer is consistent with single runs on either side
    mk = lambda M: (lambda dt: lts.Model(w.mesh, w.fine_mask, M, w.h0, w.u0, dt, w.g,
                                         precision=lts.LTS_FP32, interface_layers=layers))
    assert maxdt._stable(mk(res["M_max_stable"]), res["dt_coarse"], T, 1e-2)
    if res["tried"] and not res["tried"][-1][1]:
        M_bad = res["tried"][-1][0]
        assert not maxdt._stable(mk(M_bad), M_bad * res["dt_fine"], T, 1e-2)
