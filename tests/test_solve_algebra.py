"""The integer algebra of the GPU's exact solves, checked on the CPU.

The cluster solves split the nodes into slices and take, per slice, one block
pass of two inclusive scans (of R_k and of k R_k).  From those and the slice
prefixes A0 = sum_{k<b0} R_k, B = sum_{k<b0} k R_k they form
    P_g = A0 + I_g,  M_g = NG P_g - SP,  M_{g-1} = NG (P_g - R_g) - SP,
    sum_{k<g} P_k = g P_g - (B + J_g),
with SR = sum R_k, SP = NG SR - sum_k k R_k and M_{-1} = NG SR - SP.  These
tests check the identities exactly (Python integers) against the definitions
P_g = sum_{k<=g} R_k, M_g = NG P_g - sum_k P_k, for random slice splits, and the
resulting E and Phi (Eq. 7 and Eq. 6 in flux form) against the oracle's
direct solve.
"""
import math
import random

import numpy as np

import oracle as O


def closed_forms(R, C):
    ng = len(R)
    SR = sum(R)
    SP = ng * SR - sum(k * r for k, r in enumerate(R))
    per = (ng + C - 1) // C
    out = []
    for r in range(C):
        b0, b1 = min(ng, r * per), min(ng, r * per + per)
        A0 = sum(R[:b0])
        B = sum(k * R[k] for k in range(b0))
        I = J = 0
        for g in range(b0, b1):
            I += R[g]
            J += g * R[g]
            P = A0 + I
            M = ng * P - SP
            Mprev = ng * SR - SP if g == 0 else ng * (P - R[g]) - SP
            sumP = g * P - (B + J)
            out.append((P, M, Mprev, sumP))
    return out, SP


def definitions(R):
    ng = len(R)
    P = [sum(R[:g + 1]) for g in range(ng)]
    SPd = sum(P)
    M = [ng * p - SPd for p in P]
    Mprev = [M[g - 1] if g > 0 else M[ng - 1] for g in range(ng)]
    sumP = [sum(P[:g]) for g in range(ng)]
    return P, M, Mprev, sumP, SPd


def random_R(ng, n_per_cell, rng):
    # R_g = N 2^24 - NG rho_q[g] of an integer density with sum rho_q = N 2^24
    n = ng * n_per_cell
    total = n << 24
    cuts = sorted(rng.randrange(total + 1) for _ in range(ng - 1))
    rho_q = [b - a for a, b in zip([0] + cuts, cuts + [total])]
    return [total - ng * q for q in rho_q], n


def test_closed_forms_equal_the_definitions():
    rng = random.Random(5)
    for ng in (1, 2, 7, 64, 255, 1000):
        R, _ = random_R(ng, 50, rng)
        assert sum(R) == 0
        P, M, Mprev, sumP, SPd = definitions(R)
        for C in (1, 2, 3, 5, 16):
            got, SP = closed_forms(R, C)
            assert SP == SPd
            assert [t[0] for t in got] == P
            assert [t[1] for t in got] == M
            assert [t[2] for t in got] == Mprev
            assert [t[3] for t in got] == sumP


def test_field_from_closed_forms_matches_the_oracle():
    rng = random.Random(9)
    L = 4.0 * math.pi
    for ng in (16, 100, 512):
        R, n = random_R(ng, 30, rng)
        p = O.params(ng, n, L)
        K = 1.0 / float(n << 24)                    # rho_ion = 1
        rho = np.array([K * r for r in R])
        phi_ref, E_ref = O.field(p, rho)
        dx = L / ng
        got, SP = closed_forms(R, 4)
        E = np.array([0.5 * dx * (K / ng) * float(t[1] + t[2]) for t in got])
        phi = np.array([-dx * dx * (K / ng) * float(ng * t[3] - g * SP) for g, t in enumerate(got)])
        assert np.abs(E - E_ref).max() <= 1e-12 * max(np.abs(E_ref).max(), 1e-300)
        assert np.abs(phi - phi_ref).max() <= 1e-12 * max(np.abs(phi_ref).max(), 1e-300)
