"""Cost model on s-graded meshes (Sec. 3.5), pinned to the paper: the
special cases the construction fixes (s = 1 is a uniform mesh, q = m puts
every layer in the fine region), the derivative condition Eq. ddqS against
the speed-up Eq. speedup_det_graded it comes from (two printed formulas),
the sign statement below Eq. ddqS, the asymptotics Eq. LTSgraded_qopt and
Eq. cost_waveeq_LTSgraded2, and the worked exponents of the remark after
Cor. cor:totalcostLFgraded (d = 3, s = 2, P1: 3/8 and 17/4)."""
import math

import pytest

from paper_2106_11117_gb300 import costmodel as cm


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("m", [4, 10, 58])
def test_uniform_mesh_and_all_fine_layers_give_no_speedup(d, m):
    for q in range(1, m + 1):
        assert cm.speedup_graded(m, d, 1.0, q) == pytest.approx(1.0, rel=1e-12)
    for s in (1.5, 2.0, 3.0):
        assert cm.cost_lts_graded(m, d, s, m) == pytest.approx(cm.cost_lf_graded(m, d, s), rel=1e-12)
        assert cm.speedup_graded(m, d, s, m) == pytest.approx(1.0, rel=1e-12)
        assert cm.speedup_graded(m, d, s, 1) >= 1.0


@pytest.mark.parametrize("d,s", [(1, 2.0), (2, 2.0), (3, 2.0), (2, 3.0), (2, 1.5)])
def test_ddqS_is_the_sign_of_the_speedup_derivative(d, s):
    m = 40
    for q in (1.3, 2.0, 3.7, 6.0, 9.5, 15.0, 30.0):
        h = 1e-6 * q
        fd = (cm.speedup_graded(m, d, s, q + h) - cm.speedup_graded(m, d, s, q - h)) / (2 * h)
        lhs = cm.ddq_speedup_graded(m, d, s, q)
        g = (q + 1) ** s - q**s
        den = (m**d + q**d * (g - 1)) ** 2
        # Eq. ddqS is the derivative's numerator after dividing out m^d / den
        assert fd == pytest.approx(m**d * lhs / den, rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("d,s", [(1, 2.0), (2, 2.0), (3, 2.0), (2, 3.0)])
@pytest.mark.parametrize("m", [2, 8, 58, 464])
def test_ddqS_positive_for_small_q_and_negative_at_q_equal_m(d, s, m):
    assert cm.ddq_speedup_graded(m, d, s, 1.0) > 0 or m == 2
    assert cm.ddq_speedup_graded(m, d, s, float(m)) < 0
    q = cm.q_opt_graded(m, d, s)
    assert 1 <= q < m or m == 2


@pytest.mark.parametrize("d,s", [(1, 2.0), (2, 2.0), (3, 2.0), (2, 3.0)])
def test_optimal_layers_and_lts_cost_asymptotics(d, s):
    """q_opt = O(m^{d/(d+s-1)}) and C_LTS(q_opt) = O(m^{s + d^2/(d+s-1)}):
    the log-log slopes between m = 2^12 and 2^15 approach the exponents."""
    def slope(f):
        a, b = 2**12, 2**15
        return math.log(f(b) / f(a)) / math.log(b / a)
    q_slope = slope(lambda m: cm.q_opt_graded(m, d, s) if m < 5000 else _q_opt_fast(m, d, s))
    assert q_slope == pytest.approx(d / (d + s - 1), abs=0.03)
    c_slope = slope(lambda m: cm.cost_lts_graded(m, d, s, _q_opt_fast(m, d, s)))
    assert c_slope == pytest.approx(s + d * d / (d + s - 1), abs=0.03)


def _q_opt_fast(m, d, s):
    """argmax of the speed-up by golden-section search on [1, m] (unimodal)."""
    lo, hi = 1.0, float(m)
    r = (math.sqrt(5) - 1) / 2
    for _ in range(200):
        a, b = hi - r * (hi - lo), lo + r * (hi - lo)
        if cm.speedup_graded(m, d, s, a) < cm.speedup_graded(m, d, s, b):
            lo = a
        else:
            hi = b
    q = 0.5 * (lo + hi)
    return max((math.floor(q), math.ceil(q)), key=lambda k: cm.speedup_graded(m, d, s, max(k, 1)))


def test_remark_exponents_for_p1_in_3d_with_s_2():
    g_lf, g_lts, e = cm.graded_rates(3, 2, k=1)
    assert g_lf == 5
    assert g_lts == pytest.approx(17 / 4, rel=1e-15)
    assert e == pytest.approx(3 / 8, rel=1e-15)
    # the middle case of Eq. Qeff_graded meets the last one at beta = gamma_LTS
    assert (g_lf - g_lts) / 2 == pytest.approx(e, rel=1e-15)
