"""Pins for the oracle's post-processing: probabilities, top-k, XEB, fidelity, and the
paper's closed forms (Eqs. 1-4, App. A) against independent facts."""
import json
import math
import os

import numpy as np
import pytest

from oracle import postprocess as pp
from oracle import theory as th

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")


def test_probability_exact_values():
    a = np.array([[0.5 + 0.25j, -0.75j, 0.0]])
    p = pp.probabilities(a, 4.0)
    assert p.tolist() == [[1.25, 2.25, 0.0]]


def _brute_topk(p, idx, k):
    items = sorted(zip(p.tolist(), idx.tolist()), key=lambda t: (-t[0], t[1]))
    return [i for _, i in items[:k]], [v for v, _ in items[:k]]


@pytest.mark.parametrize("seed", range(4))
def test_topk_blocks_brute_force_with_ties(seed):
    rng = np.random.default_rng(seed)
    G, l, k = 5, 6, 9
    # amplitudes from a small set so that equal probabilities (ties) are common
    vals = np.array([0.0, 0.125, -0.125, 0.25, 0.5j, -0.25j])
    amps = vals[rng.integers(0, len(vals), size=(G, 1 << l))]
    base = np.sort(rng.choice(1 << 10, size=G, replace=False)).astype(np.int64) << 6
    pos = np.arange(l - 1, -1, -1)
    idx, p = pp.topk_blocks(amps, k, 2.0, base, pos)
    full = pp.full_indices(base, pos, l)
    for g in range(G):
        pg = (amps[g].real ** 2 + amps[g].imag ** 2) * 2.0
        ri, rp = _brute_topk(pg, full[g], k)
        assert idx[g].tolist() == ri and p[g].tolist() == rp


def test_topk_global_brute_force():
    rng = np.random.default_rng(7)
    amps = rng.normal(size=(4, 16)) + 1j * rng.normal(size=(4, 16))
    amps[1, 3] = amps[2, 5] = amps[0, 0]  # a three-way tie
    base = np.array([0, 16, 32, 48], dtype=np.int64)
    pos = np.arange(3, -1, -1)
    idx, p = pp.topk_global(amps, 10, 1.0, base, pos)
    pg = (amps.real ** 2 + amps.imag ** 2).reshape(-1)
    ri, rp = _brute_topk(pg, np.arange(64), 10)
    assert idx.tolist() == ri and p.tolist() == rp


def test_full_indices_scatter_open_bits():
    # open qubits at bit positions 5 and 1 of a 6-bit index, block base 0b010100
    idx = pp.full_indices(np.array([0b010100]), np.array([5, 1]), 2)
    assert idx.tolist() == [[0b010100, 0b010110, 0b110100, 0b110110]]


def test_xeb_definition_values():
    # Eq. (1) by hand: n = 2, q = (0.5, 0.25, 0.25, 0)
    q = np.array([0.5, 0.25, 0.25, 0.0])
    assert pp.xeb(q[[0]], 2) == 1.0
    assert pp.xeb(q[[3]], 2) == -1.0
    assert abs(pp.xeb(q, 2)) < 1e-15  # all strings: sum q = 1 -> 0


def test_xeb_of_exact_samples(sv_grid4x6):
    # samples drawn from q itself: XEB -> N sum q^2 - 1 ~ 1 for PT (Eq. 1 discussion)
    w, psi = sv_grid4x6
    N = 1 << w.n_qubits
    q = psi.real ** 2 + psi.imag ** 2
    rng = np.random.default_rng(1)
    s = rng.choice(N, size=100_000, p=q / q.sum())
    val = pp.xeb(q[s], w.n_qubits)
    expect = th.exact_sampling_xeb(float(np.sum(q * q)), N)
    assert abs(expect - 1.0) < 0.1
    assert abs(val - expect) < 0.05


def test_numerical_fidelity():
    rng = np.random.default_rng(3)
    e = rng.normal(size=64) + 1j * rng.normal(size=64)
    assert abs(pp.numerical_fidelity(3.0j * e, e) - 1.0) < 1e-14
    o = np.zeros(64, complex); o[0] = 1
    e2 = e.copy(); e2[0] = 0
    assert pp.numerical_fidelity(o, e2) == 0.0


def test_topk_xeb_order_statistics_monte_carlo():
    # E[mean of top k of m iid Exp(1)] - 1 = H_m - H_k, checked by simulation
    rng = np.random.default_rng(5)
    m, k, reps = 1024, 64, 4000
    x = rng.exponential(size=(reps, m))
    top = -np.sort(-x, axis=1)[:, :k]
    mc = float(top.mean()) - 1.0
    assert abs(mc - th.topk_xeb_exact(m, k)) < 0.01
    # and it approaches Eq. (2)'s ln(m/k)
    assert abs(th.topk_xeb_exact(m, k) - th.topk_xeb_ideal(m, k)) < 0.01


def test_appendix_tail_mass_by_quadrature():
    from scipy import integrate
    for alpha in (1e-1, 2 ** -10, 2 ** -15):
        t = th.pt_threshold(alpha)
        tail, _ = integrate.quad(lambda x: math.exp(-x), t, math.inf)
        assert abs(tail - alpha) < 1e-12
        mass, _ = integrate.quad(lambda x: x * math.exp(-x), t, math.inf)
        assert abs(mass - th.pt_tail_mass(alpha)) < 1e-12
        # XEB of the alpha fraction = mass / alpha - 1 = -ln alpha (App. A)
        assert abs(mass / alpha - 1 + math.log(alpha)) < 1e-9


def test_paper_printed_numbers():
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    # Sec. III: ln 2^15 printed as 10.3972 (k = 2^15 of 2^30)
    g = gold["topk_amplification_ln_2_15"]
    assert round(th.topk_xeb_ideal(2 ** 30, 2 ** 15), 4) == g["value"]
    # the measured ratio 10.4694 +- 0.2635 is within one sigma of the prediction
    r = gold["topk_measured_ratio"]
    assert abs(r["value"] - th.topk_xeb_ideal(2 ** 30, 2 ** 15)) < r["sigma"]


def test_topk_on_porter_thomas_blocks(sv_grid4x6):
    # per-block top-64 of 1024 exact probabilities: mean XEB ~ H_1024 - H_64 (Eq. 2, finite m)
    w, psi = sv_grid4x6
    from oracle import statevector as sv
    amps, _ = sv.block_amplitudes(psi, w.n_qubits, w.open_qubits, w.closed_qubits, w.closed_bits)
    idx, p = pp.topk_blocks(amps, 64, 1.0, w.block_base(), w.open_bit_pos())
    q = pp.ideal_probabilities_at(psi, idx)
    assert np.array_equal(q, p)  # f = 1: p is the ideal probability
    per_block = [pp.xeb(q[g], w.n_qubits) for g in range(w.G)]
    assert abs(np.mean(per_block) - th.topk_xeb_exact(1024, 64)) < 0.15


def test_table_one_arithmetic():
    # Table I: the fidelity-1 task is 2^24 sub-networks of equal cost, and the Sycamore
    # task contracts 5.5527e17 / 1.1029e14 ~ 5035 of them, i.e. ~0.03% of 2^24
    with open(GOLDEN) as fh:
        gold = json.load(fh)
    per = gold["per_subtask_complex_flop"]["value"]
    full = gold["fidelity_one_complex_flop"]["value"]
    task = gold["sycamore_task_complex_flop"]["value"]
    n = 2 ** gold["n_subtasks_log2"]["value"]
    assert abs(per * n / full - 1) < 1e-3
    frac = task / per / n * 100
    assert abs(frac - gold["fraction_of_subtasks_percent"]["value"]) < 0.0005


def test_metropolis_samples_follow_p():
    # 16 candidates with random weights (and one zero): the visit frequencies of
    # many chains converge to p / sum(p); total variation within a few
    # standard errors of the 2e5 correlated samples
    rng = np.random.default_rng(5)
    p = rng.random(16) ** 3
    p[3] = 0.0
    s = pp.metropolis(p, n_chains=2000, n_steps=120, burn=20, rng=np.random.default_rng(6))
    assert s.size == 2000 * 100
    freq = np.bincount(s, minlength=16) / s.size
    target = p / p.sum()
    assert freq[3] == 0.0  # a zero-probability candidate is never accepted
    assert 0.5 * np.abs(freq - target).sum() < 0.01, (freq, target)


def test_metropolis_xeb_of_porter_thomas_and_uniform():
    # Eq. 3 with F = 1: samples of an exponential (Porter-Thomas) q over N = 2^12
    # strings score XEB = N sum q^2 - 1 (about 1); samples of a uniform p score 0
    n = 12
    N = 1 << n
    rng = np.random.default_rng(7)
    q = rng.exponential(size=N)
    q /= q.sum()
    s = pp.metropolis(q, n_chains=4096, n_steps=64, burn=32, rng=np.random.default_rng(8))
    expect = N * float((q * q).sum()) - 1.0
    assert abs(pp.xeb(q[s], n) - expect) < 0.05, (pp.xeb(q[s], n), expect)
    assert 0.85 < expect < 1.15
    u = np.full(N, 1.0 / N)
    su = pp.metropolis(u, n_chains=512, n_steps=16, burn=4, rng=np.random.default_rng(9))
    assert abs(pp.xeb(q[su], n)) < 0.05  # uniform samples: XEB of a uniform draw ~ 0


def test_metropolis_rejects_bad_input():
    rng = np.random.default_rng(0)
    with pytest.raises(ValueError):
        pp.metropolis(np.zeros(4), 4, 4, 0, rng)
    with pytest.raises(ValueError):
        pp.metropolis(np.ones(4), 4, 4, 4, rng)
    with pytest.raises(ValueError):
        pp.metropolis(np.array([1.0, -1.0]), 4, 4, 0, rng)
