"""Host-side invariants the tensor-core kernels rely on (no GPU).

1. Work ranges of the tensor-core residual update: the (tile, chunk) units of a
   step, ntiles x nq in tile-major order, are cut into gridDim.x equal ranges
   [U b / G, U (b + 1) / G).  With G <= ntiles every range holds at least nq
   units, so a tile lies in at most two ranges; when it lies in two, it is the
   last segment of range b (its chunks from 0: part 0) and the first of range
   b + 1 (part 1), and both meet in boundary slot b.
2. Error-free slicing of the FP64 Cholesky products: a row scaled by 2^-e into
   (-1/2, 1/2) is rounded to an integer X below 2^55 and written as
   sum_p s_p 2^{56-7p} with integer |s_p| <= 64 (exact in BF16), every level
   sum of 64 slice products is an integer below 2^22 (exact in FP32), and the
   level combination reproduces the product up to the levels left out.
"""
from fractions import Fraction
import math
import random

import numpy as np


def _ranges(ntiles, nq, grid):
    U = ntiles * nq
    return [(U * b // grid, U * (b + 1) // grid) for b in range(grid)]


def test_work_ranges_split_each_tile_at_most_once():
    rng = random.Random(5)
    cases = [(2048, 32, 152), (162, 2, 152), (162, 1, 152), (152, 3, 152), (16384, 64, 152), (7, 5, 7)]
    cases += [(rng.randint(1, 3000), rng.randint(1, 64), 0) for _ in range(300)]
    for ntiles, nq, grid in cases:
        grid = grid or rng.randint(1, min(ntiles, 200))
        owners = {}
        for b, (u0, u1) in enumerate(_ranges(ntiles, nq, grid)):
            assert u1 - u0 >= nq  # every range holds a whole tile's worth of chunks
            u = u0
            while u < u1:
                tile, q = divmod(u, nq)
                q_last = min(nq - 1, q + (u1 - u) - 1)
                owners.setdefault(tile, []).append((b, q, q_last))
                u += q_last - q + 1
        assert sorted(owners) == list(range(ntiles))
        for tile, parts in owners.items():
            assert len(parts) in (1, 2)
            if len(parts) == 1:
                assert parts[0][1:] == (0, nq - 1)  # whole tile
            else:
                (b0, qa0, qb0), (b1, qa1, qb1) = parts
                assert b1 == b0 + 1  # neighbouring ranges share it: boundary slot b0
                assert qa0 == 0 and qb1 == nq - 1 and qa1 == qb0 + 1


def _slices(v, e):
    """Integer slices of v 2^-e (|v| 2^-e < 1/2): X = round(v 2^{56-e}), s_p, p = 1..8."""
    X = int(round(Fraction(v) * Fraction(2) ** (56 - e)))
    assert abs(X) < 2 ** 55
    s, t = [], X
    for p in range(1, 9):
        sft = 56 - 7 * p
        sp = (t + (1 << (sft - 1))) >> sft if sft > 0 else t  # round half up, as the kernel
        t -= sp << sft
        s.append(sp)
    assert t == 0 and sum(sp << (56 - 7 * p) for p, sp in enumerate(s, 1)) == X
    return s


def test_slice_products_are_exact_and_close_to_the_fp64_product():
    rng = np.random.default_rng(11)
    K = 64
    for trial in range(40):
        spread = [0.0, 4.0, 20.0][trial % 3]  # entries of similar size, or spread over 2^20
        a = rng.standard_normal(K) * np.exp2(rng.uniform(-spread, 0, K))
        c = rng.standard_normal(K) * np.exp2(rng.uniform(-spread, 0, K))
        ea = max(math.frexp(x)[1] for x in a) + 1  # |a| 2^-ea < 1/2
        ec = max(math.frexp(x)[1] for x in c) + 1
        sa = [_slices(x, ea) for x in a]
        sc = [_slices(x, ec) for x in c]
        for row in sa + sc:
            assert all(abs(s) <= 64 for s in row)
        acc = {}
        for L in range(2, 10):
            tot = 0
            for p in range(max(1, L - 8), min(8, L - 1) + 1):
                q = L - p
                tot += sum(sa[kk][p - 1] * sc[kk][q - 1] for kk in range(K))
            assert abs(tot) < 2 ** 22  # exact in the FP32 accumulators
            acc[L] = tot
        H = sum(acc[L] * 2 ** (7 * (5 - L)) for L in range(2, 6))
        Lo = sum(acc[L] * 2 ** (7 * (9 - L)) for L in range(6, 10))
        assert abs(H) < 2 ** 51 and abs(Lo) < 2 ** 51  # exact through the FP64 mantissa
        # the kernel: t = fl(Lo 2^-28 + H), product = t 2^{ea+ec-35}
        t = math.fma(float(Lo), 2.0 ** -28, float(H)) if hasattr(math, "fma") else float(Fraction(Lo, 2 ** 28) + H)
        got = Fraction(t) * Fraction(2) ** (ea + ec - 35)
        exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a, c))
        bound = Fraction(2) ** -50 * K * Fraction(max(abs(a))) * Fraction(max(abs(c))) * 8 \
            + Fraction(abs(float(exact))) * Fraction(2) ** -52
        assert abs(got - exact) <= bound, float(abs(got - exact) / bound)


def _tc_constants():
    """The pipeline constants of the tensor-core update, read from its source."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2310_17137_gb300", "csrc", "kmv_tc.cu")).read()
    vals = {}
    for name in ("kRows", "kChunk", "kStages", "kBufs", "kColsPerWarp", "kSlots", "kTcMaxKdp"):
        m = re.search(r"constexpr int %s = (\d+);" % name, src)
        assert m, name
        vals[name] = int(m.group(1))
    vals["kGroups"] = vals["kChunk"] // vals["kColsPerWarp"]
    return vals


def _slot_chunks(slot, n_slots, n_groups, n_chunks):
    """Chunks of the work items of one transform warp: items c * n_groups + g, taken
    round-robin by the n_slots warps of a lane quarter starting at their slot."""
    return [i // n_groups for i in range(slot, n_chunks * n_groups, n_slots)]


def _max_gap(n_slots, n_groups, n_chunks=64):
    gaps = []
    for s in range(n_slots):
        ch = _slot_chunks(s, n_slots, n_groups, n_chunks)
        assert ch[0] < n_groups and all(b >= a for a, b in zip(ch, ch[1:]))
        gaps += [b - a for a, b in zip(ch, ch[1:])]
    return max(gaps)


def test_transform_schedule_keeps_buffer_phases_unambiguous():
    # A transform warp waits on the S barrier of its item's buffer by phase parity.
    # Its previous item's S was complete, and the distance MMAs complete in chunk
    # order, so the buffer has completed at least the phase of chunk c - kBufs as
    # long as consecutive items of a warp are at most kBufs chunks apart; it cannot
    # complete the phase after c before this warp's P of chunk c is consumed.
    k = _tc_constants()
    items = sorted(i for s in range(k["kSlots"]) for i in range(s, 64 * k["kGroups"], k["kSlots"]))
    assert items == list(range(64 * k["kGroups"]))  # every item of a quarter exactly once
    assert _max_gap(k["kSlots"], k["kGroups"]) <= k["kBufs"]
    # the rule is not vacuous: thirteen warps per quarter would skip a whole ring
    assert _max_gap(13, k["kGroups"]) > k["kBufs"]


def test_tensor_core_update_fits_tmem_and_shared_memory():
    k = _tc_constants()
    for C in (16, 32):
        assert k["kBufs"] * k["kChunk"] + 3 * C <= 512  # S/P ring + three accumulators
    kdp, C = k["kTcMaxKdp"], 32
    xa = k["kRows"] * kdp * 2
    stage = k["kChunk"] * kdp * 2 + 2 * C * k["kChunk"] * 2
    assert 2 * xa + k["kStages"] * stage + 1024 <= 227 * 1024 - 8 * 1024  # dynamic + static headroom
