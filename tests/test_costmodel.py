"""Cost models of MLMC with leapfrog and with LF-LTS (Sec. 3.2-3.4), pinned to
what the paper fixes: the per-level costs of one dQ_l sample (Eq. C_l_LTS and
the level terms of Eq. fullQ_eff) when the refinement factor halves per level
(p_l = p_0 / 2^l, H_l = H_0 / 2^l), the closed form of the speed-up S (Prop.
3.2, Eq. fullQ_eff), and the statements of Sec. 3.4 about where the speed-up
peaks (Table tab:Q_eff parameters; single solve at r = 1/100^d)."""
import math

import pytest

from paper_2106_11117_gb300 import costmodel as cm


def _paper_level_terms(d, r, p0, l):
    """Bracketed level terms of Eq. fullQ_eff (costs in units of T k^{2(d+1)} / H_0^{d+1})."""
    if l == 0:
        return (1 - r) * p0 + r * p0 ** (d + 1), (1 - r) + r * p0 ** (d + 1)
    lf = r * 2 * p0 ** (d + 1) + (1 - r) * 2 ** ((d + 1) * l) * (2**d + 1) / 2 ** (d + l) * p0
    lts = r * 2 * p0 ** (d + 1) + (1 - r) * 2 ** ((d + 1) * l) * (2 ** (d + 1) + 1) / 2 ** (d + 1)
    return lf, lts


@pytest.mark.parametrize("d", [1, 2, 3])
@pytest.mark.parametrize("r,p0", [(1e-2, 13.0), (1e-4, 19.0), (0.3, 4.0)])
def test_level_costs_match_the_papers_level_terms(d, r, p0):
    L = 4
    p_levels = [p0 / 2**l for l in range(L + 1)]
    lf = cm.level_costs(1.0, 1, d, 1.0, p_levels, r, "lf")
    lts = cm.level_costs(1.0, 1, d, 1.0, p_levels, r, "lts")
    for l in range(L + 1):
        a, b = _paper_level_terms(d, r, p0, l)
        assert lf[l] == pytest.approx(a, rel=1e-12)
        assert lts[l] == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("d,r,p0,beta", [(1, 1e-2, 13.0, 4), (2, 1e-4, 19.0, 6), (3, 1e-6, 27.0, 8), (2, 0.05, 8.0, 2)])
def test_speedup_matches_prop_3_2(d, r, p0, beta):
    L = 5
    V = [3.0 * 2.0 ** (-beta * l) for l in range(L + 1)]
    p_levels = [p0 / 2**l for l in range(L + 1)]
    S = cm.speedup_S(V, cm.level_costs(2.0, 3, d, 0.5, p_levels, r, "lf"),
                     cm.level_costs(2.0, 3, d, 0.5, p_levels, r, "lts"))
    num = math.fsum(math.sqrt(V[l] * _paper_level_terms(d, r, p0, l)[0]) for l in range(L + 1))
    den = math.fsum(math.sqrt(V[l] * _paper_level_terms(d, r, p0, l)[1]) for l in range(L + 1))
    assert S == pytest.approx((num / den) ** 2, rel=1e-12)


@pytest.mark.parametrize("d", [1, 2, 3])
def test_single_solve_speedup_peaks_between_10_and_30(d):
    """Sec. 3.4: the speed-up of one LTS solve over leapfrog (Eq.
    cost_waveeq_LF over Eq. cost_waveeq_LTS) at r = 1/100^d is largest for
    p between 10 and 30."""
    r = 1.0 / 100**d
    ratio = {p: cm.cost_lf(1, 1, d, 1, p, r) / cm.cost_lts(1, 1, d, 1, p, r) for p in range(1, 400)}
    best = max(ratio, key=ratio.get)
    assert 10 <= best <= 30
    assert ratio[best] > ratio[5] and ratio[best] > ratio[60]


@pytest.mark.parametrize("d,r,beta", [(1, 1e-2, 4), (2, 1e-4, 6), (3, 1e-6, 8)])
def test_mlmc_speedup_peaks_between_10_and_30(d, r, beta):
    """Sec. 3.4 with Table tab:Q_eff: L = ceil(log2 p_0) levels, p_l = p_0/2^l
    on levels 0..L-1 and a uniform finest level (p_L = 1), V_l = V_0 2^{-beta l};
    for fixed r the speed-up S is largest for p_0 between 10 and 30 and
    smaller again for larger p_0."""
    S = {}
    for p0 in range(2, 121):
        L = math.ceil(math.log2(p0))
        p_levels = [p0 / 2**l for l in range(L)] + [1.0]
        V = [2.0 ** (-beta * l) for l in range(L + 1)]
        S[p0] = cm.speedup_S(V, cm.level_costs(1, 1, d, 1, p_levels, r, "lf"),
                             cm.level_costs(1, 1, d, 1, p_levels, r, "lts"))
    best = max(S, key=S.get)
    assert 10 <= best <= 30
    assert S[120] < S[best] and S[4] < S[best]


def test_speedup_approaches_the_coarsest_level_ratio_for_small_r():
    """Sec. 3.4: as r decreases the speed-up grows until it reaches the
    speed-up of LTS over leapfrog on the coarsest level, here p_0 (level 0
    carries the cost when V_l decays fast)."""
    d, p0 = 2, 16.0
    p_levels = [p0 / 2**l for l in range(5)]
    V = [2.0 ** (-30 * l) for l in range(5)]
    prev = 0.0
    for r in (1e-1, 1e-2, 1e-3, 1e-4, 1e-6, 1e-9):
        S = cm.speedup_S(V, cm.level_costs(1, 1, d, 1, p_levels, r, "lf"),
                         cm.level_costs(1, 1, d, 1, p_levels, r, "lts"))
        assert S > prev
        prev = S
    assert prev == pytest.approx(p0, rel=1e-3)


def test_speedup_is_a_ratio_of_costs():
    V = [1.0, 0.3, 0.05, 0.01]
    C = [1.0, 5.0, 21.0, 90.0]
    assert cm.speedup_S(V, [2.5 * c for c in C], C) == pytest.approx(2.5, rel=1e-14)
    assert cm.speedup_S([7 * v for v in V], [2.5 * c for c in C], C) == pytest.approx(2.5, rel=1e-14)
    assert cm.speedup_S(V, C, C) == pytest.approx(1.0, rel=1e-14)


def test_solve_work_counts_dof_updates():
    """Eq. cost_waveeq_LTS in DOF updates: one update per free DOF per step
    plus p updates of each DOF of R; leapfrog at dt/p updates every DOF p
    times per coarse step; with nothing refined (R empty) they differ by p."""
    assert cm.solve_work(100, 1000, 200, 8, "lts") == 100 * (1000 + 8 * 200)
    assert cm.solve_work(100, 1000, 200, 8, "lf") == 8 * 100 * 1000
    assert cm.solve_work(100, 1000, 0, 8, "lf") == 8 * cm.solve_work(100, 1000, 0, 8, "lts")
