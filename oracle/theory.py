"""Closed forms from arXiv 2406.18889 (test infrastructure only).

* Porter-Thomas (Sec. III, App. A): for deep random circuits the scaled
  probability x = N q is distributed as P(x) = e^{-x}.
* Ideal top-k XEB (Eq. 2, App. A): keeping the k largest of |S~| PT
  probabilities gives <F_XEB> = ln(|S~|/k).  In App. A the threshold printed as
  "t = ln N/k" is read as t = ln(N/k), with N the number of candidates, and the
  kept mass is int_t^inf x e^{-x} dx = alpha (1 - ln alpha), alpha = k/N.
* Approximate top-k XEB (Eq. 4): F ln(|S~|/k) at simulation fidelity F, with
  F = f for a fraction f of the sub-networks (Eq. 3).
* Finite-size exact form: for m iid Exp(1) draws the mean of the k largest is
  1 + H_m - H_k (order statistics), so the ideal top-k XEB is H_m - H_k, which
  tends to ln(m/k) for large m and k.
"""
from __future__ import annotations

import math


def harmonic(m: int) -> float:
    return math.fsum(1.0 / j for j in range(1, m + 1))


def topk_xeb_exact(m: int, k: int) -> float:
    """E[F_XEB] of the top k of m iid Porter-Thomas probabilities: H_m - H_k."""
    return harmonic(m) - harmonic(k)


def topk_xeb_ideal(n_candidates: float, k: float) -> float:
    """Eq. (2): ln(|S~| / k)."""
    return math.log(n_candidates / k)


def topk_xeb_approx(F: float, n_candidates: float, k: float) -> float:
    """Eq. (4): F ln(|S~| / k)."""
    return F * math.log(n_candidates / k)


def pt_threshold(alpha: float) -> float:
    """App. A: t with int_t^inf e^{-x} dx = alpha, i.e. t = ln(1/alpha)."""
    return -math.log(alpha)


def pt_tail_mass(alpha: float) -> float:
    """App. A: int_t^inf x e^{-x} dx at that threshold = alpha (1 - ln alpha)."""
    return alpha * (1.0 - math.log(alpha))


def haar_second_moment(N: int) -> float:
    """E[(N q)^2] over a Haar-random state of dimension N: 2N/(N+1)."""
    return 2.0 * N / (N + 1.0)


def exact_sampling_xeb(q_sum_sq: float, N: int) -> float:
    """Expected F_XEB of samples drawn from q itself: N sum_s q(s)^2 - 1."""
    return N * q_sum_sq - 1.0
