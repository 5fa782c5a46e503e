"""Invariants of the slice GEMM's tile schedule, checked on a model of its index arithmetic (CPU).

The tensor-core kernel relies on properties of the passes the host builds, for every slice count
up to 8:
- every pass has slices lo = 0 .. hi = the pass's top level;
- A tile j of a K-step (slice hi - j) is last used together with B_j, so both leave through one
  shared ring slot;
- the producers' copy order (per B_j: the A tiles down to the lowest slice B_j meets, then B_j)
  never has to wait for a slot that only a later MMA would free, with 6 slots per operand;
- a pass's K-chunk keeps every FP32 level sum an exact integer (< 2^24) for any input.
This model restates those rules to check them for all shapes; the GPU tests check the kernel."""
import pytest

NS = 6          # ring slots per operand
BETA = 7        # digit width: |digit| <= 2^(BETA-1), so a product is at most 2^(2 BETA - 2)


def host_groups(s):
    """Level groups as the host builds them: pairs {L-1, L} from the top level s-1 down."""
    groups = []
    L = s - 1
    while L >= 0:
        groups.append((L - 1, 2) if L >= 1 else (0, 1))
        L -= 2
    return groups


def slice_range(glo, gn, s):
    L1, L2 = glo, glo + gn - 1
    return max(0, L1 - (s - 1)), min(L2, s - 1)


def exact_chunk(glo, gn, s):
    """Longest K-chunk (a multiple of 64) whose level sums stay below 2^24."""
    q = max(min(L, s - 1) - max(0, L - s + 1) + 1 for L in range(glo, glo + gn))
    per = 1 << (2 * BETA - 2)
    return max(64, ((1 << 24) // (q * per)) // 64 * 64)


SHAPES = [(s, glo, gn) for s in range(1, 9) for glo, gn in host_groups(s)]


@pytest.mark.parametrize("s,glo,gn", SHAPES)
def test_pass_shape_is_lockstep(s, glo, gn):
    lo, hi = slice_range(glo, gn, s)
    L1, L2 = glo, glo + gn - 1
    assert lo == 0 and hi == L2
    last_use = {}
    for j in range(lo, hi + 1):
        for L in range(L1, L2 + 1):
            i = L - j
            if lo <= i <= hi:
                last_use[hi - i] = j  # A FIFO position of slice i
    # every A position is used, and position k is last used at step k, with B_k
    assert sorted(last_use) == list(range(hi - lo + 1))
    assert all(last_use[k] == k for k in last_use)


@pytest.mark.parametrize("s,glo,gn", SHAPES)
def test_exact_chunk_bounds_level_sums(s, glo, gn):
    kc = exact_chunk(glo, gn, s)
    assert kc % 64 == 0
    for L in range(glo, glo + gn):
        q = min(L, s - 1) - max(0, L - s + 1) + 1  # products in level L
        assert q * (1 << (2 * BETA - 2)) * kc <= 1 << 24


def simulate(passes, ksteps):
    """Run the producers' copy order against a 6-slot ring per operand, releasing A position j
    and B_j after step j; returns the number of steps completed (a stall would end early)."""
    seq = []  # (kind, index in that operand's sequence, step it belongs to)
    steps = []  # per step: (A tiles needed through, B index)
    na = nb = 0
    for glo, gn, s in passes:
        lo, hi = slice_range(glo, gn, s)
        L1 = glo
        for _ in range(ksteps):
            a_base = na
            a_here = 0
            for j in range(lo, hi + 1):
                imin = max(L1 - j, lo)
                while a_here < hi - imin + 1:
                    seq.append(("A", na))
                    na += 1
                    a_here += 1
                seq.append(("B", nb))
                steps.append((a_base + (hi - imin), nb, a_base + (j - lo)))
                nb += 1
    released_a = released_b = 0  # tiles released so far (in order)
    loaded = {"A": 0, "B": 0}
    done = 0
    pos = 0
    progress = True
    while progress:
        progress = False
        # producers: load while the slot's previous use has been released
        while pos < len(seq):
            kind, u = seq[pos]
            rel = released_a if kind == "A" else released_b
            if u - NS >= 0 and u - NS >= rel:
                break
            loaded[kind] = u + 1
            pos += 1
            progress = True
        # issuer: run the next step if its tiles have landed
        while done < len(steps):
            a_need, b_idx, a_free = steps[done]
            if loaded["A"] <= a_need or loaded["B"] <= b_idx:
                break
            # release A position j and B_j together (in sequence order)
            released_a = max(released_a, a_free + 1)
            released_b = b_idx + 1
            done += 1
            progress = True
    return done, len(steps)


@pytest.mark.parametrize("s", range(1, 9))
def test_ring_never_stalls(s):
    passes = [(glo, gn, s) for glo, gn in host_groups(s)]
    done, total = simulate(passes * 2, ksteps=5)
    assert done == total
