"""Planted mistakes: each test copies an oracle source file, plants one plausible mistake (a
dropped term, a flipped sign, a wrong index, a transposed operand), and checks that one of the
pins of ``test_oracle_qb.py`` / ``test_oracle_philox.py`` now fails.  Everything runs on the CPU
against the oracle only."""
import os
import sys
import types

import numpy as np
import pytest

import synth

ORACLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")


def mutated(fname: str, old: str, new: str) -> types.ModuleType:
    src = open(os.path.join(ORACLE, fname)).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    src = src.replace(old, new).replace("from .philox import", "from oracle.philox import")
    mod = types.ModuleType("oracle_mutant_" + fname.replace(".py", ""))
    sys.modules[mod.__name__] = mod  # dataclasses look their module up
    exec(compile(src, fname + ":mutant", "exec"), mod.__dict__)
    return mod


def prop2_gap(mod) -> float:
    A = synth.dense_from_spectrum(90, 70, synth.sigma_exp(70, 8.0), seed=11)
    r_fp = mod.randqb_fp(A, 0.0, 5, seed=4, fixed_rank=20)
    r_ei = mod.randqb_ei(A, 0.0, 5, seed=4, fixed_rank=20)
    return np.linalg.norm(r_fp.Q @ r_fp.B - r_ei.Q @ r_ei.B) / np.linalg.norm(A)


def thm1_gap(mod) -> float:
    A = synth.dense_from_spectrum(64, 48, synth.sigma_exp(48, 6.0), seed=2)
    r = mod.randqb_ei(A, 1e-5, 5, seed=7)
    worst = 0.0 if len(r.E_hist) == r.rank else np.inf
    for k in range(1, min(r.rank, len(r.E_hist)) + 1):
        direct = np.linalg.norm(A - r.Q[:, :k] @ r.B[:k]) ** 2
        worst = max(worst, abs(r.E_hist[k - 1] - direct) / r.normA2)
    return worst


@pytest.mark.parametrize("old,new", [
    ("- Om_i.T @ (B.T @ B)\n            else", "+ Om_i.T @ (B.T @ B)\n            else"),  # sign
    ("Bi = np.linalg.solve(Ri.T, S)", "Bi = np.linalg.solve(Ri, S)"),                   # R^-1 vs R^-T
    ("S = H[:, c0:c0 + bi].T - (Y.T @ Q)", "S = H[:, 0:bi].T - (Y.T @ Q)"),               # block index
])
def test_planted_fp_mistakes_break_proposition2(old, new):
    import oracle.qb as good
    assert prop2_gap(good) <= 1e-10
    assert prop2_gap(mutated("qb.py", old, new)) > 1e-6


@pytest.mark.parametrize("old,new", [
    ("E = E - float(np.dot(Bi[j], Bi[j]))", "E = E - float(np.dot(Bi[j], Bi[j - 1]))"),  # index
    ("return E, j + 1, True", "return E, j, True"),                                        # off by one
])
def test_planted_indicator_mistakes_break_theorem1(old, new):
    import oracle.qb as good
    assert thm1_gap(good) <= 1e-12
    assert thm1_gap(mutated("qb.py", old, new)) > 1e-8


def test_planted_relative_criterion_mistake_breaks_table4_pin():
    mod = mutated("qb.py", "return tol * np.sqrt(normA2) if relative else tol",
                  "return tol * normA2 if relative else tol")
    n = 400
    sigma = synth.table4_matrix_spectra(n)["M1"]
    A = 37.5 * synth.dense_from_spectrum(n, n, sigma, seed=42)
    r = mod.randqb_ei(A, 1e-2, 10, seed=1, P=1)
    r_svd = synth.svd_rank(sigma, 1e-2)
    err = np.linalg.norm(A - r.Q @ r.B) / np.linalg.norm(A)
    assert not (err < 1e-2 and r_svd <= r.rank <= r_svd + 3)


@pytest.mark.parametrize("old,new", [
    ("C = np.tril(M) + np.tril(M, -1).T", "C = np.triu(M) + np.triu(M, 1).T"),
    ("return Q @ GB + Ybar @ Om.T", "return Q @ GB"),
    ("Qbar = GQ + A @ GB.T", "Qbar = GQ"),
])
def test_planted_adjoint_mistakes_break_finite_differences(old, new):
    mod = mutated("qb.py", old, new)
    m, n, k = 48, 36, 6
    A = synth.dense_from_spectrum(m, n, synth.sigma_pow(36, 1.0), seed=4)
    GQ, GB = synth.cotangents(m, n, k, seed=5)
    Abar = mod.qb_fixed_rank_adjoint(A, k, 7, GQ, GB)
    V = np.random.default_rng(0).standard_normal((m, n))
    h = 1e-6

    def loss(X):
        Q, B, _ = mod.qb_fixed_rank(X, k, 7)
        return float(np.sum(GQ * Q) + np.sum(GB * B))

    fd = (loss(A + h * V) - loss(A - h * V)) / (2 * h)
    assert abs(fd - float(np.sum(Abar * V))) > 1e-4 * abs(fd)


@pytest.mark.parametrize("old,new", [
    ("p1 = m1 * c2", "p1 = m1 * c3"),
    ("k0 = np.uint64((int(k0) + W0) & MASK32)", "k0 = np.uint64((int(k0) + W1) & MASK32)"),
])
def test_planted_philox_mistakes_break_known_answers(old, new):
    mod = mutated("philox.py", old, new)
    out = mod.philox4x32_10(0, 0, 0, 0, 0, 0)
    assert [int(x) for x in out] != [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def test_planted_box_muller_mistake_breaks_pairing():
    mod = mutated("philox.py", "rho * np.cos(theta), rho * np.sin(theta))\n\n\ndef omega_f32",
                  "rho * np.cos(theta), rho * np.cos(theta))\n\n\ndef omega_f32")
    z = mod.omega(50000, 0, 2, seed=9402)
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) > 0.5


def test_planted_h_from_sketch_copy_breaks_b_equals_qta():
    """randQB_FP must form H = A^T G from A itself; H taken from the sketch copy makes B differ
    from Q^T A by about the copy's rounding."""
    A = synth.dense_from_spectrum(300, 200, synth.sigma_exp(200, 20.0, 1e-6), seed=31)
    As = A + 1e-3 * np.linalg.norm(A) / np.sqrt(A.size) * \
        np.random.default_rng(0).standard_normal(A.shape)

    def gap(mod):
        r = mod.randqb_fp(A, 1e-3, 10, seed=3, P=1, A_sketch=As)
        return np.linalg.norm(r.B - r.Q.T @ A) / np.linalg.norm(A)

    import oracle.qb as good
    assert gap(good) <= 1e-10
    assert gap(mutated("qb.py", "H = np.asarray(A.T @ G)", "H = np.asarray(As.T @ G)")) > 1e-6
