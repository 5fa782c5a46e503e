"""Pins for the FP64 CPU oracle: values and identities fixed by the paper's
definitions and by mathematics, none of them produced by the oracle itself.

R[i,j,a,b] = sum_cd (sum_P L_Pac L_Pbd) t_ijcd   (Eq. 5 + Eq. 6)

Each pin is chosen so that a plausible slip in the oracle fails at least one:
a transposed L index (L_Pca for L_Pac) fails the rank-1 and single-entry pins
with non-symmetric L; a c<->d swap (the exchange term of Eq. 7) fails the
single-entry pin; a dropped P term fails the identity / Cholesky-batch pins;
a wrong output index fails the golden fixture.
"""
import json
import os

import numpy as np
import pytest

from paper_2310_04559_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- golden case
def test_golden_terms_hand_computed(oracle):
    """Eq. 7, Eq. 8 and Eq. 9 on a hand-computed case (derivation in the fixture)."""
    g = json.load(open(os.path.join(GOLDEN, "terms_o1_v2_n2.json")))
    L = np.array(g["L"], dtype=float)
    t2 = np.array(g["t2"], dtype=float)
    Lov = np.array(g["Lov"], dtype=float)
    assert np.array_equal(oracle.exchange(L, t2), np.array(g["X"], dtype=float))
    assert np.array_equal(oracle.tijkl(Lov, t2), np.array(g["tijkl"], dtype=float))
    assert np.array_equal(oracle.tijbk(Lov, L, t2), np.array(g["tijbk"], dtype=float))


def test_golden_hand_computed(oracle):
    g = json.load(open(os.path.join(GOLDEN, "ladder_o1_v2_n2.json")))
    L = np.array(g["L"], dtype=float)
    t2 = np.array(g["t2"], dtype=float)
    W = np.array(g["W"], dtype=float)
    R = oracle.ladder(L, t2)
    assert np.array_equal(R, np.array(g["R"], dtype=float))
    assert np.array_equal(oracle.ladder_eri(L, t2), np.array(g["R"], dtype=float))
    assert oracle.energy(R, t2) == g["E"]
    dL, dt2 = oracle.ladder_grad(L, t2, W)
    assert np.array_equal(dt2, np.array(g["dt2"], dtype=float))
    assert np.array_equal(dL, np.array(g["dL"], dtype=float))
    assert float(np.sum(W * R)) == g["loss"]


# ------------------------------------------------------------- brute force
@pytest.mark.parametrize("o,v,n,sym", [(1, 1, 1, False), (2, 3, 5, False), (3, 7, 11, False),
                                       (4, 24, 60, True), (2, 13, 9, False)])
def test_bruteforce_eri(oracle, o, v, n, sym):
    """a-loop oracle == explicit dense (ac|bd) tensor contracted over (c,d)."""
    rng = np.random.default_rng(o * 100 + v)
    L = synth.cholesky_vectors(n, v, symmetric=sym, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=sym, rng=rng)
    R = oracle.ladder(L, t2)
    assert _rel(R, oracle.ladder_eri(L, t2)) < 1e-14


def test_paper_einsum_string(oracle):
    """Section 3.1 one-shot contraction "xac,xbd,icjd->iajb" (paper layout
    t[i,c,j,d]) evaluated by numpy.einsum, a third-party implementation."""
    o, v, n = 3, 9, 17
    L = _rand((n, v, v), 3)
    t2 = _rand((o, o, v, v), 4)
    t_paper = t2.transpose(0, 2, 1, 3)  # [i,c,j,d]
    R_paper = np.einsum("xac,xbd,icjd->iajb", L, L, t_paper, optimize=True)
    R = oracle.ladder(L, t2)
    assert _rel(R, R_paper.transpose(0, 2, 1, 3)) < 1e-13


# ------------------------------------------------------------- closed forms
def test_identity_vector_gives_t(oracle):
    """n = 1, L_0 = I  =>  (ac|bd) = delta_ac delta_bd  =>  R = t2 exactly."""
    o, v = 3, 6
    t2 = _rand((o, o, v, v), 5)
    R = oracle.ladder(np.eye(v)[None], t2)
    assert np.array_equal(R, t2)


def test_scaled_identities(oracle):
    """L_P = alpha_P I  =>  R = (sum_P alpha_P^2) t2."""
    o, v = 2, 5
    alpha = np.array([0.5, -2.0, 0.25])
    L = alpha[:, None, None] * np.eye(v)[None]
    t2 = _rand((o, o, v, v), 6)
    assert _rel(oracle.ladder(L, t2), np.sum(alpha ** 2) * t2) < 1e-15


def test_rank_one_outer_product(oracle):
    """L_0 = x y^T (non-symmetric)  =>  R_ijab = x_a x_b (y^T t_ij y)."""
    o, v = 3, 7
    x, y = _rand(v, 7), _rand(v, 8)
    L = np.outer(x, y)[None]
    t2 = _rand((o, o, v, v), 9)
    s = np.einsum("c,ijcd,d->ij", y, t2, y)
    ref = s[:, :, None, None] * np.outer(x, x)[None, None]
    assert _rel(oracle.ladder(L, t2), ref) < 1e-13


def test_single_amplitude_gives_integral_column(oracle):
    """t_ij,cd = delta_(ij,c0 d0)  =>  R_ij,ab = (a c0 | b d0) = sum_P L_P,a,c0 L_P,b,d0
    for that (i,j) and zero elsewhere; c0 != d0 and non-symmetric L separate
    the direct term from the exchange term of Eq. 7."""
    o, v, n = 2, 6, 4
    L = _rand((n, v, v), 10)
    c0, d0 = 1, 4
    t2 = np.zeros((o, o, v, v))
    t2[1, 0, c0, d0] = 1.0
    R = oracle.ladder(L, t2)
    col = sum(np.outer(L[P][:, c0], L[P][:, d0]) for P in range(n))
    assert _rel(R[1, 0], col) < 1e-15
    assert not R[0].any() and not R[1, 1].any()


# --------------------------------------------------------------- invariants
def test_pair_symmetry_any_L(oracle):
    """t_ijcd = t_jidc  =>  R_ijab = R_jiba for ANY L (swap c<->d in the sum)."""
    o, v, n = 3, 8, 6
    L = _rand((n, v, v), 11)  # not symmetric in (a,c)
    t2 = synth.amplitudes(o, v, rng=np.random.default_rng(12))
    R = oracle.ladder(L, t2)
    assert _rel(R, R.transpose(1, 0, 3, 2)) < 1e-14


def test_linear_in_t_quadratic_in_L(oracle):
    o, v, n = 2, 6, 5
    L = _rand((n, v, v), 13)
    t, u = _rand((o, o, v, v), 14), _rand((o, o, v, v), 15)
    R = oracle.ladder(L, 2.0 * t - 3.0 * u)
    assert _rel(R, 2.0 * oracle.ladder(L, t) - 3.0 * oracle.ladder(L, u)) < 1e-13
    assert _rel(oracle.ladder(-1.5 * L, t), 2.25 * oracle.ladder(L, t)) < 1e-14


def test_cholesky_batches_add_and_rotate(oracle):
    """R(L1 (+) L2) = R(L1) + R(L2); R is invariant under permutations and
    orthogonal rotations Q of the Cholesky index (same integrals, Eq. 5)."""
    o, v = 2, 6
    L1, L2 = _rand((4, v, v), 16), _rand((3, v, v), 17)
    t2 = _rand((o, o, v, v), 18)
    L = np.concatenate([L1, L2])
    R = oracle.ladder(L, t2)
    assert _rel(R, oracle.ladder(L1, t2) + oracle.ladder(L2, t2)) < 1e-13
    assert _rel(oracle.ladder(L[::-1].copy(), t2), R) < 1e-13
    Q, _ = np.linalg.qr(_rand((7, 7), 19))
    Lq = np.einsum("QP,Pac->Qac", Q, L)
    assert _rel(oracle.ladder(Lq, t2), R) < 1e-12


def test_exchange_is_direct_with_cd_swapped(oracle):
    """Eq. 7: sum_cd (ad|bc) t_ijcd = sum_cd (ac|bd) t_ijdc."""
    o, v, n = 2, 7, 5
    L, t2 = _rand((n, v, v), 20), _rand((o, o, v, v), 21)
    X = oracle.exchange(L, t2)
    assert _rel(X, oracle.ladder(L, np.ascontiguousarray(t2.transpose(0, 1, 3, 2)))) < 1e-13
    assert _rel(X, np.einsum("xad,xbc,ijcd->ijab", L, L, t2)) < 1e-13
    sub = oracle.exchange(L, t2, a_list=[4, 0])
    assert np.array_equal(sub, X[:, :, [4, 0], :])


def test_a_list_sampling_and_compensation(oracle):
    o, v, n = 3, 10, 12
    L, t2 = synth.ladder_inputs(o, v, n, seed=22)
    R = oracle.ladder(L, t2)
    al = [7, 0, 9, 3]
    assert np.array_equal(oracle.ladder(L, t2, a_list=al), R[:, :, al, :])
    Rc = oracle.ladder(L, t2, compensated=True)
    assert _rel(R, Rc) < 1e-14


def test_entries_match_the_full_term(oracle):
    """Entries computed one by one are the full term's entries bit for bit (same sums in the
    same order) and agree with the brute force through the dense integral tensor; a transposed
    L (non-symmetric here) or a swapped (a, b) would fail."""
    o, v, n = 3, 11, 9
    rng = np.random.default_rng(24)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=False, rng=rng)
    R = oracle.ladder(L, t2)
    idx = np.concatenate([rng.integers(0, R.size, 40), [0, R.size - 1]])
    assert np.array_equal(oracle.ladder_entries(L, t2, idx), R.ravel()[idx])
    assert _rel(oracle.ladder_entries(L, t2, idx), oracle.ladder_eri(L, t2).ravel()[idx]) < 1e-14
    assert oracle.ladder_entries(L, t2, []).size == 0


# ----------------------------------------------------------------- energy
def test_energy_hand_and_identities(oracle):
    # o = v = 1: E = (2R - R) t = R t = (sum_P L_P^2) t^2
    L = np.array([[[2.0]], [[-3.0]]])
    t2 = np.array([[[[0.5]]]])
    R = oracle.ladder(L, t2)
    assert R[0, 0, 0, 0] == 13.0 * 0.5
    assert oracle.energy(R, t2) == 13.0 * 0.25
    o, v, n = 3, 6, 7
    L, t2 = synth.ladder_inputs(o, v, n, seed=23)
    R = oracle.ladder(L, t2)
    E, ep = oracle.energy(R, t2, pair=True)
    ref = 2.0 * np.vdot(R, t2) - np.vdot(R.transpose(0, 1, 3, 2), t2)
    assert abs(E - ref) <= 1e-13 * abs(ref)
    assert abs(ep.sum() - E) <= 1e-13 * abs(E)
    # symmetric t: the exchange-like part equals sum R_jiab t_ijab
    assert abs(np.vdot(R.transpose(0, 1, 3, 2), t2) - np.vdot(R.transpose(1, 0, 2, 3), t2)) < 1e-13 * abs(E)


def test_energy_range_shares(oracle):
    """One part's share of E under an `a`-range partition: the terms with min(a, b) in [lo, hi).
    Pinned by hand for o = 1, v = 2, by the full range, and by additivity over a partition."""
    R = np.array([[[[1.0, 2.0], [3.0, 5.0]]]])
    t2 = np.array([[[[7.0, 11.0], [13.0, 17.0]]]])
    # min(a, b) = 0: (a, b) = (0,0), (0,1), (1,0);  min = 1: (1,1) only
    e0 = (2 * 1 - 1) * 7 + (2 * 2 - 3) * 11 + (2 * 3 - 2) * 13
    e1 = (2 * 5 - 5) * 17
    assert oracle.energy_range(R, t2, 0, 1) == e0
    assert oracle.energy_range(R, t2, 1, 2) == e1
    assert oracle.energy_range(R, t2, 0, 2) == oracle.energy(R, t2) == e0 + e1
    o, v, n = 3, 9, 7
    L, t2 = synth.ladder_inputs(o, v, n, seed=29)
    R = oracle.ladder(L, t2)
    E = oracle.energy(R, t2)
    assert abs(oracle.energy_range(R, t2, 0, v) - E) <= 1e-14 * abs(E)
    for cuts in ([0, 4, 9], [0, 1, 2, 5, 9], [0, 8, 9]):
        parts = sum(oracle.energy_range(R, t2, cuts[g], cuts[g + 1]) for g in range(len(cuts) - 1))
        assert abs(parts - E) <= 1e-13 * abs(E), cuts
    assert oracle.energy_range(R, t2, 3, 3) == 0.0


# --------------------------------------------------------------- gradient
def test_gradient_identities_and_fd(oracle):
    o, v, n = 2, 5, 4
    rng = np.random.default_rng(24)
    L = _rand((n, v, v), 25)  # general (non-symmetric) L
    t2 = _rand((o, o, v, v), 26)
    W = synth.cotangent(o, v, rng=rng)
    dL, dt2 = oracle.ladder_grad(L, t2, W)
    loss = float(np.sum(W * oracle.ladder(L, t2)))
    assert abs(np.vdot(dt2, t2) - loss) < 1e-12 * abs(loss)          # linear in t2
    assert abs(np.vdot(dL, L) - 2.0 * loss) < 1e-12 * abs(loss)     # degree 2 in L
    h = 1e-6
    for k in range(12):
        idx = tuple(rng.integers(0, s) for s in L.shape)
        Lp, Lm = L.copy(), L.copy()
        Lp[idx] += h
        Lm[idx] -= h
        fd = (np.sum(W * oracle.ladder(Lp, t2)) - np.sum(W * oracle.ladder(Lm, t2))) / (2 * h)
        assert abs(fd - dL[idx]) < 1e-7 * (1 + abs(dL[idx]))
        jdx = tuple(rng.integers(0, s) for s in t2.shape)
        tp, tm = t2.copy(), t2.copy()
        tp[jdx] += h
        tm[jdx] -= h
        fd = (np.sum(W * oracle.ladder(L, tp)) - np.sum(W * oracle.ladder(L, tm))) / (2 * h)
        assert abs(fd - dt2[jdx]) < 1e-7 * (1 + abs(dt2[jdx]))


def test_gradient_adjoint_forms_and_entries(oracle):
    """dt2 = ladder(L^T, W) with L^T_Pac = L_Pca (and = ladder(L, W) for
    symmetric L); for symmetric t, dL = T1[W] + T1[W^swap] collapses onto the
    first sum alone evaluated with W + W^swap."""
    o, v, n = 2, 6, 5
    L = _rand((n, v, v), 27)
    t2 = _rand((o, o, v, v), 28)
    W = _rand((o, o, v, v), 29)
    dL, dt2 = oracle.ladder_grad(L, t2, W)
    assert _rel(dt2, oracle.ladder(np.ascontiguousarray(L.transpose(0, 2, 1)), W)) < 1e-13
    Ls = synth.cholesky_vectors(n, v, rng=np.random.default_rng(30))
    _, dts = oracle.ladder_grad(Ls, t2, W)
    assert _rel(dts, oracle.ladder(Ls, W)) < 1e-13
    # one-by-one entries equal the full arrays
    rng = np.random.default_rng(31)
    i1 = rng.integers(0, dt2.size, 9)
    i2 = rng.integers(0, dL.size, 9)
    e1, e2 = oracle.ladder_grad_entries(L, t2, W, i1, i2)
    assert np.array_equal(e1, dt2.ravel()[i1]) or _rel(e1, dt2.ravel()[i1]) < 1e-15
    assert _rel(e2, dL.ravel()[i2]) < 1e-15


# ------------------------------------------------- Eq. 8 and Eq. 9 (two-block terms)
# tt_ijkl = sum_{P,c,d} L^P_kc L^P_ld t_ij^cd and tt_ijbk = sum_{P,c,d} L^P_bd L^P_kc t_ij^cd share
# the ladder's contraction.  Pins: reduction to the pinned ladder when the occupied-virtual block is
# part of the virtual-virtual one, rank-one closed forms that separate every index, the pair
# symmetry of Eq. 8, and additivity over Cholesky batches.  A swapped output pair (k <-> l, b <-> k),
# a c <-> d swap or an L_ck for L_kc fails at least one of them.

def _terms_inputs(o, v, n, seed):
    rng = np.random.default_rng(seed)
    Lvv = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    Lov = synth.cholesky_ov(n, o, v, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=False, rng=rng)
    return Lov, Lvv, t2


@pytest.mark.parametrize("o,v,n", [(2, 5, 3), (3, 7, 11), (4, 9, 6)])
def test_terms_reduce_to_the_ladder(oracle, o, v, n):
    """With Lov[P,k,c] = L[P,k,c] for k < o (o <= v), Eq. 8 is the ladder's R[i,j,k,l] and Eq. 9
    is R[i,j,k,b] read as tt[i,j,b,k]."""
    _, L, t2 = _terms_inputs(o, v, n, 40 + o)
    R = oracle.ladder(L, t2)
    Lov = np.ascontiguousarray(L[:, :o, :])
    assert _rel(oracle.tijkl(Lov, t2), R[:, :, :o, :o]) < 1e-14
    assert _rel(oracle.tijbk(Lov, L, t2), R[:, :, :o, :].transpose(0, 1, 3, 2)) < 1e-14


def test_terms_rank_one_closed_forms(oracle):
    """n = 1, Lov[0] = x y^T, Lvv[0] = u w^T:
    tt_ijkl = x_k x_l (y^T t_ij y),  tt_ijbk = u_b x_k (y^T t_ij w)."""
    o, v = 3, 6
    rng = np.random.default_rng(44)
    x, y = rng.standard_normal(o), rng.standard_normal(v)
    u, w = rng.standard_normal(v), rng.standard_normal(v)
    t2 = rng.standard_normal((o, o, v, v))
    Lov = np.outer(x, y)[None]
    Lvv = np.outer(u, w)[None]
    s_yy = np.array([[y @ t2[i, j] @ y for j in range(o)] for i in range(o)])
    s_yw = np.array([[y @ t2[i, j] @ w for j in range(o)] for i in range(o)])
    ref1 = s_yy[:, :, None, None] * np.outer(x, x)[None, None]
    ref2 = s_yw[:, :, None, None] * np.outer(u, x)[None, None]
    assert _rel(oracle.tijkl(Lov, t2), ref1) < 1e-14
    assert _rel(oracle.tijbk(Lov, Lvv, t2), ref2) < 1e-14


def test_terms_pair_symmetry_and_batches(oracle):
    """Eq. 8 inherits the pair symmetry: t_ijcd = t_jidc gives tt_ijkl = tt_jilk for any Lov.
    Both terms are additive over concatenated Cholesky batches."""
    o, v, n = 4, 8, 10
    rng = np.random.default_rng(45)
    Lov = synth.cholesky_ov(n, o, v, rng=rng)
    Lvv = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    ts = synth.amplitudes(o, v, symmetric=True, rng=rng)
    T = oracle.tijkl(Lov, ts)
    assert _rel(T, T.transpose(1, 0, 3, 2)) < 1e-14
    t2 = synth.amplitudes(o, v, symmetric=False, rng=rng)
    for f in (lambda a, b: oracle.tijkl(a, t2), lambda a, b: oracle.tijbk(a, b, t2)):
        whole = f(Lov, Lvv)
        parts = f(Lov[:4], Lvv[:4]) + f(Lov[4:], Lvv[4:])
        assert _rel(parts, whole) < 1e-13
