"""Pins for the oracle's Maxwell-Boltzmann-scaling (MBS) thermostat (reading R22).

The thermostat rescales each cell's velocities relative to the cell's centre of mass so that
their kinetic energy becomes kT times a Gamma(3/2 (n_c - 1)) draw: the canonical distribution
of the relative kinetic energy of n_c particles, which has 3 (n_c - 1) quadratic degrees of
freedom (Huang et al. 2010, the cell-level thermostat the paper cites in Sec. 2 and Sec. 4).
The draw uses Marsaglia and Tsang's rejection method.

What pins it, independently of the oracle's own code:
  * the draws follow scipy's Gamma distribution (Kolmogorov-Smirnov, mean, variance);
  * after a thermostatted step, every cell's relative kinetic energy, mapped through the
    Gamma CDF of its own n_c, is uniform on [0, 1] (pooled over all cells and steps);
  * momentum is conserved cell by cell, and the rule is deterministic in (seed, step, cell).
"""
import numpy as np
import pytest
from scipy import stats

from paper_2212_11878_gb300 import inputs


@pytest.mark.parametrize("shape", [1.5, 3.0, 13.5, 28.5])
def test_mbs_gamma_follows_gamma_distribution(orc, shape):
    p = orc.make_params((4, 4, 4), seed=4242)
    x = np.array([orc.mbs_gamma(p, t, c, shape) for t in range(1, 21) for c in range(1000)])
    n = x.size
    assert stats.kstest(x, stats.gamma(shape).cdf).pvalue > 1e-3
    assert abs(x.mean() - shape) < 5 * np.sqrt(shape / n)
    # var of the sample variance of Gamma(a): (mu4 - sigma^4)/n with mu4 = 3a^2 + 6a
    assert abs(x.var() - shape) < 5 * np.sqrt((3 * shape ** 2 + 6 * shape - shape ** 2) / n)


def test_mbs_gamma_is_a_function_of_seed_step_cell(orc):
    p = orc.make_params((4, 4, 4), seed=11)
    q = orc.make_params((4, 4, 4), seed=12)
    a = orc.mbs_gamma(p, 5, 17, 13.5)
    assert orc.mbs_gamma(p, 5, 17, 13.5) == a
    assert orc.mbs_gamma(p, 6, 17, 13.5) != a
    assert orc.mbs_gamma(p, 5, 18, 13.5) != a
    assert orc.mbs_gamma(q, 5, 17, 13.5) != a


def test_mbs_thermostat_gives_canonical_cell_energies(orc):
    L = (16, 16, 16)
    kT = 1.7
    p = orc.make_params(L, thermostat=2, kT=kT, seed=31)
    n = int(round(10 * np.prod(L)))
    r, v = inputs.uniform_gaussian_state(L, n, 32, kT=kT)
    st = orc.State(r, v)
    C = orc.num_cells(p)
    pits = []
    for _ in range(3):
        out = orc.step(p, st, debug=True)
        keys = out["keys"]
        cnt = np.bincount(keys, minlength=C)
        P = np.stack([np.bincount(keys, weights=st.v[:, d], minlength=C) for d in range(3)], axis=1)
        assert np.abs(P - out["moments"][:, 1:4]).max() < 1e-12 * 30       # momentum per cell
        u = P / np.maximum(cnt, 1)[:, None]
        rel = 0.5 * np.bincount(keys, weights=((st.v - u[keys]) ** 2).sum(axis=1), minlength=C)
        ok = cnt >= 2
        pits.append(stats.gamma.cdf(rel[ok] / kT, 1.5 * (cnt[ok] - 1)))
    pit = np.concatenate(pits)
    assert stats.kstest(pit, "uniform").pvalue > 1e-3


def test_mbs_and_rescale_agree_on_the_mean(orc):
    """The deterministic rescale (R14) sets every cell to the mean of the MBS target."""
    L = (12, 12, 12)
    n = int(round(10 * np.prod(L)))
    r, v = inputs.uniform_gaussian_state(L, n, 33)
    tot = {}
    for th in (1, 2):
        p = orc.make_params(L, thermostat=th, seed=34)
        st = orc.State(r, v)
        out = orc.step(p, st, debug=True)
        keys = out["keys"]
        C = orc.num_cells(p)
        cnt = np.bincount(keys, minlength=C)
        u = np.stack([np.bincount(keys, weights=st.v[:, d], minlength=C) for d in range(3)], axis=1)
        u /= np.maximum(cnt, 1)[:, None]
        rel = 0.5 * np.bincount(keys, weights=((st.v - u[keys]) ** 2).sum(axis=1), minlength=C)
        tot[th] = rel[cnt >= 2].sum()
        dof = (1.5 * (cnt[cnt >= 2] - 1)).sum()
    assert abs(tot[1] / dof - 1) < 1e-12
    assert abs(tot[2] / dof - 1) < 5 / np.sqrt(dof)
