"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative Frobenius error ||R - R_oracle|| / ||R_oracle||):
  fp64        1e-12   DMMA with FP64 accumulation: error ~ sqrt(K) * 2^-53
  ozaki_bf16  1e-10   6 slices x 7 bits = 42 bits per operand; exact FP32 slice products
  tf32        1e-2    10-bit mantissa inputs, FP32 accumulation per K-chunk
  bf16        5e-2    7-bit mantissa inputs
"""
import numpy as np
import pytest
import torch

from paper_2310_04559_gb300 import binding as B
from paper_2310_04559_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "ozaki_bf16": 1e-10, "tf32": 1e-2, "bf16": 5e-2}
MODES = list(TOL)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda", 0)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cu(x, dev):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


# ------------------------------------------------------------- GEMM core
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (37, 300, 70), (200, 513, 1000), (129, 257, 4100)])
def test_gemm_core(dev, mode, M, N, K):
    rng = np.random.default_rng(M + N + K)
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-3, 3, (M, 1)))
    Bm = rng.standard_normal((N, K))
    ref = A @ Bm.T
    C = B.gemm(cu(A, dev), cu(Bm, dev), mode=mode).cpu().numpy()
    assert rel(C, ref) < TOL[mode], (mode, rel(C, ref))
    # accumulate adds into C
    C2 = B.gemm(cu(A, dev), cu(Bm, dev), mode=mode, C=cu(ref, dev), accumulate=True).cpu().numpy()
    assert rel(C2, 2 * ref) < TOL[mode]


def test_gemm_ozaki_exact_integers(dev):
    """Integer inputs that fit in the leading slice give the exact product."""
    rng = np.random.default_rng(5)
    A = rng.integers(-40, 41, (130, 300)).astype(np.float64)
    Bm = rng.integers(-40, 41, (270, 300)).astype(np.float64)
    C = B.gemm(cu(A, dev), cu(Bm, dev), mode="ozaki_bf16").cpu().numpy()
    assert np.array_equal(C, A @ Bm.T)


# ------------------------------------------------------------ ladder forward
def _fwd(L, t2, dev, **kw):
    R = B.ladder_forward(cu(L, dev), cu(t2, dev), **kw)
    if isinstance(R, tuple):
        return R[0].cpu().numpy(), float(R[1].cpu())
    return R.cpu().numpy()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("order", ["integral_first", "cholesky_first"])
def test_tiny_workload_all_modes(dev, oracle, mode, order):
    o, v, n = 4, 24, 60
    L, t2 = synth.ladder_inputs(o, v, n, seed=0)
    R_ref = oracle.ladder(L, t2)
    for sym in (False, True):
        R = _fwd(L, t2, dev, mode=mode, order=order, symmetric=sym)
        assert rel(R, R_ref) < TOL[mode], (mode, order, sym, rel(R, R_ref))


@pytest.mark.parametrize("mode", MODES)
def test_ragged_multiblock(dev, oracle, mode):
    """Shapes that span several tiles with ragged tails, non-symmetric L and t2,
    and forced small a-blocks (ragged last block)."""
    o, v, n = 5, 37, 150
    rng = np.random.default_rng(11)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=False, rng=rng)
    R_ref = oracle.ladder(L, t2)
    for order in ("integral_first", "cholesky_first"):
        for ab in (0, 7):
            R = _fwd(L, t2, dev, mode=mode, order=order, a_block=ab)
            assert rel(R, R_ref) < TOL[mode], (order, ab, rel(R, R_ref))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("a_block", [0, 7, 1])
def test_pair_symmetric_ragged_blocks(dev, oracle, mode, a_block):
    """Pair-symmetric t2 with a non-symmetric L (the kernels may use (ac|bd) = (bd|ac),
    never L_Pac = L_Pca): ragged tiles, forced small a-blocks and one `a` per block, so
    the b >= a integral blocks, the c <= d packing and the four-way write of R meet
    every diagonal case."""
    o, v, n = 5, 37, 150
    rng = np.random.default_rng(31)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=True, rng=rng)
    R_ref = oracle.ladder(L, t2)
    R = _fwd(L, t2, dev, mode=mode, symmetric=True, a_block=a_block, order="integral_first")
    assert rel(R, R_ref) < TOL[mode], (mode, a_block, rel(R, R_ref))
    if mode != "fp64":
        # R[i,j,a,b] and R[j,i,b,a] are written from one value
        assert np.array_equal(R, R.transpose(1, 0, 3, 2))


@pytest.mark.parametrize("o,v,n", [(1, 9, 5), (3, 1, 4), (2, 2, 3), (1, 1, 1), (6, 65, 17)])
def test_pair_symmetric_degenerate_shapes(dev, oracle, o, v, n):
    """o = 1 (no i < j pairs), v = 1 (no c < d entries), and tiny shapes."""
    rng = np.random.default_rng(o * 100 + v)
    L = synth.cholesky_vectors(n, v, symmetric=False, rng=rng)
    t2 = synth.amplitudes(o, v, symmetric=True, rng=rng)
    R_ref = oracle.ladder(L, t2)
    for mode in ("ozaki_bf16", "tf32"):
        R = _fwd(L, t2, dev, mode=mode, symmetric=True)
        assert rel(R, R_ref) < TOL[mode], (mode, rel(R, R_ref))


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_flags_accumulate_exchange_energy(dev, oracle, mode):
    o, v, n = 3, 29, 41
    L, t2 = synth.ladder_inputs(o, v, n, seed=3)
    R_ref = oracle.ladder(L, t2)
    X_ref = oracle.exchange(L, t2)
    E_ref = oracle.energy(R_ref, t2)
    R0 = np.random.default_rng(4).standard_normal(t2.shape)
    for sym in (False, True):
        R = B.ladder_forward(cu(L, dev), cu(t2, dev), R=cu(R0, dev), mode=mode, symmetric=sym,
                             accumulate=True).cpu().numpy()
        assert rel(R - R0, R_ref) < 10 * TOL[mode]
        X = _fwd(L, t2, dev, mode=mode, symmetric=sym, exchange=True)
        assert rel(X, X_ref) < TOL[mode]
        R, E = _fwd(L, t2, dev, mode=mode, symmetric=sym, energy=True)
        assert abs(E - E_ref) / abs(E_ref) < TOL[mode]
    Eg, ep = B.pair_energy(cu(R_ref, dev), cu(t2, dev), pairs=True)
    E1, ep1 = oracle.energy(R_ref, t2, pair=True)
    assert abs(float(Eg.cpu()) - E1) <= 1e-13 * abs(E1)
    assert np.allclose(ep.cpu().numpy(), ep1, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_closed_forms_on_device(dev, mode):
    """L_0 = I (n = 1) gives R = t2; a rank-one L gives an outer product."""
    o, v = 3, 33
    t2 = np.random.default_rng(6).standard_normal((o, o, v, v))
    R = _fwd(np.eye(v)[None], t2, dev, mode=mode)
    assert rel(R, t2) < TOL[mode]
    x, y = np.random.default_rng(7).standard_normal((2, v))
    s = np.einsum("c,ijcd,d->ij", y, t2, y)
    ref = s[:, :, None, None] * np.outer(x, x)[None, None]
    R = _fwd(np.outer(x, y)[None], t2, dev, mode=mode)
    assert rel(R, ref) < TOL[mode]


def test_workload_o20_v200_n1000_sampled(dev, oracle):
    """Full-size o=20, v=200, n=1000 in FP64 and emulated FP64, both orders,
    checked on sampled `a` columns the oracle computes one by one."""
    o, v, n = 20, 200, 1000
    L, t2 = synth.ladder_inputs(o, v, n, seed=0)
    al = [0, 77, 199]
    R_ref = oracle.ladder(L, t2, a_list=al)
    for mode in ("fp64", "ozaki_bf16"):
        for order in ("integral_first", "cholesky_first"):
            R = _fwd(L, t2, dev, mode=mode, order=order, symmetric=True, budget=24 << 30)
            assert rel(R[:, :, al, :], R_ref) < TOL[mode], (mode, order)
            assert rel(R, R.transpose(1, 0, 3, 2)) < 1e-15 + TOL[mode]


def test_workload_o40_v400_n2000_sampled(dev, oracle):
    """The o=40, v=400, n=2000 benchmark workload in the launch configuration the
    benchmark times (emulated FP64, pair-symmetric packed path, workspace sized to a
    150 GB device budget, no status sync in the call): sampled `a` columns against the
    oracle, the pair symmetry of the whole R, and the pair energy against the oracle's
    reduction of the same R within the rounding bound of an FP64 sum of 2.6e8 terms."""
    o, v, n = 40, 400, 2000
    L, t2 = synth.ladder_inputs(o, v, n, seed=0)
    Lg, tg = cu(L, dev), cu(t2, dev)
    budget = int(150e9) - L.nbytes - 2 * t2.nbytes - (2 << 30)
    ws = B.alloc_workspace(B.workspace_size(o, v, n, mode="ozaki_bf16", symmetric=True, budget=budget), dev)
    R = torch.empty_like(tg)
    B.ladder_forward(Lg, tg, R=R, mode="ozaki_bf16", symmetric=True, workspace=ws, no_sync=True)
    from paper_2310_04559_gb300 import _lib
    _lib.check(_lib.load().cc_ladder_device_status(B._ptr(ws), B._stream(dev)), "o40 forward")
    E = float(B.pair_energy(R, tg))
    Rh = R.cpu().numpy()
    del Lg, tg, R, ws
    torch.cuda.empty_cache()
    al = [0, 199, 399]
    assert rel(Rh[:, :, al, :], oracle.ladder(L, t2, a_list=al)) < TOL["ozaki_bf16"]
    assert rel(Rh, Rh.transpose(1, 0, 3, 2)) < 1e-15
    terms = (2.0 * Rh - Rh.transpose(0, 1, 3, 2)) * t2
    assert abs(E - oracle.energy(Rh, t2)) <= 1e-14 * float(np.abs(terms).sum())


def test_workload_o60_v600_n3000_sampled_entries(dev, oracle):
    """The largest workload (o=60, v=600, n=3000: 15 blocks of `a` under a 150 GB device
    budget) in emulated FP64 with pair symmetry: 32 entries R[i,j,a,b] against the oracle's
    entries computed one by one (the full oracle would take hours), scaled by the norm of the
    sampled oracle values, and R[i,j,a,b] = R[j,i,b,a] at the same places."""
    o, v, n = 60, 600, 3000
    L, t2 = synth.ladder_inputs(o, v, n, seed=0)
    Lg, tg = cu(L, dev), cu(t2, dev)
    budget = int(150e9) - L.nbytes - 2 * t2.nbytes - (2 << 30)
    ws = B.alloc_workspace(B.workspace_size(o, v, n, mode="ozaki_bf16", symmetric=True, budget=budget), dev)
    R = torch.empty_like(tg)
    B.ladder_forward(Lg, tg, R=R, mode="ozaki_bf16", symmetric=True, workspace=ws)
    rng = np.random.default_rng(60)
    i, j, a, b = (rng.integers(0, m, 32) for m in (o, o, v, v))
    # include the corners and the diagonal cases of the four-way write
    i[:4], j[:4], a[:4], b[:4] = [0, o - 1, 5, 7], [0, o - 1, 5, 9], [0, v - 1, 11, 13], [0, v - 1, 11, 2]
    idx = ((i * o + j) * v + a) * v + b
    mirror = ((j * o + i) * v + b) * v + a
    flat = R.view(-1)
    got = flat[torch.from_numpy(idx).to(dev)].cpu().numpy()
    got_m = flat[torch.from_numpy(mirror).to(dev)].cpu().numpy()
    del Lg, tg, R, ws, flat
    torch.cuda.empty_cache()
    ref = oracle.ladder_entries(L, t2, idx)
    assert rel(got, ref) < TOL["ozaki_bf16"]
    assert np.array_equal(got, got_m)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_adjoint_vs_oracle(dev, oracle, mode):
    o, v, n = 3, 14, 23
    rng = np.random.default_rng(8)
    L = rng.standard_normal((n, v, v))
    t2 = rng.standard_normal((o, o, v, v))
    W = rng.standard_normal((o, o, v, v))
    dL_ref, dt2_ref = oracle.ladder_grad(L, t2, W)
    dL, dt2 = B.ladder_backward(cu(L, dev), cu(t2, dev), cu(W, dev), mode=mode)
    assert rel(dt2.cpu().numpy(), dt2_ref) < TOL[mode]
    assert rel(dL.cpu().numpy(), dL_ref) < TOL[mode]
    # pair-symmetric t: one dL pass with W + W^swap
    ts = synth.amplitudes(o, v, rng=rng)
    dL_ref, dt2_ref = oracle.ladder_grad(L, ts, W)
    dL, dt2 = B.ladder_backward(cu(L, dev), cu(ts, dev), cu(W, dev), mode=mode, symmetric=True)
    assert rel(dt2.cpu().numpy(), dt2_ref) < TOL[mode]
    assert rel(dL.cpu().numpy(), dL_ref) < TOL[mode]


def test_adjoint_autograd_identities(dev):
    o, v, n = 4, 20, 30
    L, t2 = synth.ladder_inputs(o, v, n, seed=9)
    W = synth.cotangent(o, v, seed=10)
    Lg, tg = cu(L, dev).requires_grad_(), cu(t2, dev).requires_grad_()
    R = B.ladder(Lg, tg, mode="fp64", symmetric=True)
    loss = (R * cu(W, dev)).sum()
    loss.backward()
    lv = float(loss.detach())
    assert abs(float((tg.grad * tg).sum()) - lv) < 1e-11 * abs(lv)
    assert abs(float((Lg.grad * Lg).sum()) - 2 * lv) < 1e-11 * abs(lv)


def test_adjoint_workload_o16_v160_n800(dev, oracle):
    """Full-size adjoint workload in FP64 through the autograd.Function: sampled
    gradient entries against the oracle computed one by one, directional central
    finite differences (h = 1e-6; the loss is linear in t2 and quadratic in L, so
    central differences are exact up to rounding), and the emulated-FP64 adjoint."""
    o, v, n = 16, 160, 800
    L, t2 = synth.ladder_inputs(o, v, n, seed=4)
    W = synth.cotangent(o, v, seed=5)
    Wg = cu(W, dev)
    Lg, tg = cu(L, dev).requires_grad_(), cu(t2, dev).requires_grad_()
    R = B.ladder(Lg, tg, mode="fp64", symmetric=True)
    (R * Wg).sum().backward()
    dL, dt2 = Lg.grad.detach(), tg.grad.detach()
    rng = np.random.default_rng(6)
    i1 = rng.integers(0, t2.size, 24)
    i2 = rng.integers(0, L.size, 24)
    e1, e2 = oracle.ladder_grad_entries(L, t2, W, i1, i2)
    assert np.allclose(dt2.cpu().numpy().ravel()[i1], e1, rtol=1e-11, atol=1e-13 * np.abs(e1).max())
    assert np.allclose(dL.cpu().numpy().ravel()[i2], e2, rtol=1e-11, atol=1e-13 * np.abs(e2).max())

    def loss(Lx, tx):
        return float((B.ladder_forward(Lx, tx, mode="fp64", symmetric=True) * Wg).sum())

    h = 1e-6
    Lc, tc = cu(L, dev), cu(t2, dev)
    for seed in (7, 8):
        DL = cu(np.random.default_rng(seed).standard_normal(L.shape), dev)
        fd = (loss(Lc + h * DL, tc) - loss(Lc - h * DL, tc)) / (2 * h)
        an = float((dL * DL).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)
        Dt = cu(synth.amplitudes(o, v, rng=np.random.default_rng(seed + 10), sigma=1.0), dev)
        fd = (loss(Lc, tc + h * Dt) - loss(Lc, tc - h * Dt)) / (2 * h)
        an = float((dt2 * Dt).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)
    # emulated FP64 adjoint agrees with the FP64 one
    dLz, dtz = B.ladder_backward(Lc, tc, Wg, mode="ozaki_bf16", symmetric=True)
    assert rel(dtz.cpu().numpy(), dt2.cpu().numpy()) < 1e-10
    assert rel(dLz.cpu().numpy(), dL.cpu().numpy()) < 1e-10


@pytest.mark.parametrize("mode", ["fp64", "ozaki_bf16"])
def test_a_range_shards_assemble(dev, oracle, mode):
    """Disjoint a-ranges (one per device in a multi-GPU run, from the work-balanced partition that
    bench.py uses) write disjoint entries; their sum is the full R, with and without pair
    symmetry, and on the pair-symmetric path the ranges' energy shares add up to the energy."""
    o, v, n = 4, 45, 70
    L, t2 = synth.ladder_inputs(o, v, n, seed=12)
    Lg, tg = cu(L, dev), cu(t2, dev)
    R_ref = oracle.ladder(L, t2)
    for sym in (False, True):
        # integral-first: the pair-symmetric path whose ranges own their energy terms
        full = B.ladder_forward(Lg, tg, mode=mode, symmetric=sym, order="integral_first")
        bounds = B.partition(o, v, n, 3, mode=mode, symmetric=sym, order="integral_first")
        assert bounds[0] == 0 and bounds[-1] == v
        parts = torch.zeros_like(full)
        e_sum = 0.0
        for g in range(3):
            lo, hi = bounds[g], bounds[g + 1]
            Rp = torch.zeros_like(full)
            if sym:
                _, Eg = B.ladder_forward(Lg, tg, R=Rp, mode=mode, symmetric=sym, a_range=(lo, hi), energy=True,
                                         order="integral_first")
                e_g = float(Eg)
                assert abs(e_g - oracle.energy_range(R_ref, t2, lo, hi)) <= TOL[mode] * abs(oracle.energy(R_ref, t2))
                e_sum += e_g
            else:
                B.ladder_forward(Lg, tg, R=Rp, mode=mode, symmetric=sym, a_range=(lo, hi), order="integral_first")
            # nothing outside this range's share is written
            parts += Rp
        assert rel(parts.cpu().numpy(), full.cpu().numpy()) < 1e-14
        assert rel(parts.cpu().numpy(), R_ref) < TOL[mode]
        if sym:
            E = oracle.energy(R_ref, t2)
            assert abs(e_sum - E) <= TOL[mode] * abs(E)


@pytest.mark.parametrize("n", [7000, 20000])
def test_long_cholesky_contraction(dev, oracle, n):
    """n_chol beyond 6144: the integral builds split K across CTAs (2 and 4 splits) so that every
    FP32 level sum stays exact.  L without decay and amplitudes diagonal in (c, d) make
    R[i,j,a,a] = sum_c (ac|ac) t_ijcc, built only from diagonal integrals, whose lower-digit squares
    add with one sign (without the split their level sums pass 2^24 near n = 12 000)."""
    o, v = 2, 10
    rng = np.random.default_rng(n)
    L = synth.cholesky_vectors(n, v, decay=0.0, rng=rng)
    tau = rng.standard_normal((o, o, v))
    tau = 0.5 * (tau + tau.transpose(1, 0, 2))  # t_ijcc = t_jicc (pair symmetry)
    t2 = np.zeros((o, o, v, v))
    t2[:, :, np.arange(v), np.arange(v)] = tau
    R_ref = oracle.ladder(L, t2)
    diag = np.arange(v)
    for mode in ("fp64", "ozaki_bf16"):
        R = _fwd(L, t2, dev, mode=mode, symmetric=True, order="integral_first")
        assert rel(R, R_ref) < TOL[mode], (mode, rel(R, R_ref))
        assert rel(R[:, :, diag, diag], R_ref[:, :, diag, diag]) < TOL[mode]
    # the Eq. 8 term's integral build and the adjoint's take the same split
    Lov = np.ascontiguousarray(L[:, :o, :])
    T = B.tijkl(cu(Lov, dev), cu(t2, dev), mode="ozaki_bf16").cpu().numpy()
    assert rel(T, oracle.tijkl(Lov, t2)) < TOL["ozaki_bf16"]
    if n == 7000:
        W = rng.standard_normal((o, o, v, v))
        dL_ref, dt2_ref = oracle.ladder_grad(L, t2, W)
        dL, dt2 = B.ladder_backward(cu(L, dev), cu(t2, dev), cu(W, dev), mode="ozaki_bf16", symmetric=True)
        assert rel(dt2.cpu().numpy(), dt2_ref) < TOL["ozaki_bf16"]
        assert rel(dL.cpu().numpy(), dL_ref) < TOL["ozaki_bf16"]
