"""The exactness rule of the complex64 top-k's reduced mode, on the CPU.

Each warp scans its own contiguous slice and keeps only its best kw
candidates; the blocks and the final pass merge what the warps kept.  The
rule: the merged top k equals the true top k unless some slice holds kw of
the merged result (then the call reruns with kw = k).  Reason: an element of
the true top k that its warp dropped is beaten by all kw entries that warp
kept, so those kw are in the true top k too, and, since the merged result
then differs from the true one only below them, in the merged result.  The
simulation uses the kernel's total order (p descending, index ascending)."""
import numpy as np
import pytest


def order(p, idx):
    return np.lexsort((idx, -p))


def true_topk(p, k):
    return order(p, np.arange(p.size))[:k]


def reduced_topk(p, k, kw, slice_len):
    kept = []
    for lo in range(0, p.size, slice_len):
        seg = np.arange(lo, min(lo + slice_len, p.size))
        kept.append(seg[order(p[seg], seg)[:kw]])
    cand = np.concatenate(kept)
    return cand[order(p[cand], cand)[:k]]


def suspect(result, slice_len, kw):
    _, counts = np.unique(result // slice_len, return_counts=True)
    return bool(np.any(counts >= kw))


@pytest.mark.parametrize("seed", range(40))
def test_rule_never_passes_a_wrong_result(seed):
    rng = np.random.default_rng(seed)
    n_amp, slice_len, kw = 1 << 14, 256, 16
    k = int(rng.choice([17, 32, 64, 128]))
    p = rng.exponential(1.0, n_amp)
    if seed % 3 == 1:   # a cluster of peaks inside one slice
        s = int(rng.integers(0, n_amp // slice_len)) * slice_len
        p[s:s + int(rng.integers(5, 60))] += 50 + rng.random()
    if seed % 3 == 2:   # heavy ties: coarse quantisation
        p = np.round(p, 1)
    got = reduced_topk(p, k, kw, slice_len)
    want = true_topk(p, k)
    if not suspect(got, slice_len, kw):
        assert list(got) == list(want)


def test_both_outcomes_occur_and_suspect_cases_can_be_wrong():
    """the rule is not vacuous: a cluster makes the reduced result wrong,
    and the rule flags it; spread inputs pass it"""
    rng = np.random.default_rng(1)
    n_amp, slice_len, kw, k = 1 << 14, 256, 16, 64
    p = rng.exponential(1.0, n_amp)
    assert not suspect(reduced_topk(p, k, kw, slice_len), slice_len, kw)
    p[512:552] += 100.0
    got = reduced_topk(p, k, kw, slice_len)
    assert suspect(got, slice_len, kw)
    assert list(got) != list(true_topk(p, k))
