"""Pins of the profile-HMM oracle (oracle/hmm.c) against brute force and closed
forms: alignment distance by enumerating every alignment, the Viterbi and
Forward scores by enumerating every state path, the profile of identical
training sequences in closed form, and the counts of single insertions and
deletions.  Then the
library's host-side profile builder against the pinned oracle (no GPU)."""
import math

import numpy as np
import pytest

import oracle

LET = "ACGT"


def _brute_distance(s: str, r: str) -> int:
    """Minimum cost over every alignment path (moves: diagonal, consume s, consume r)."""
    best = None

    def cost(a, b):
        return 0 if (a == b and a in LET) else 1

    def walk(i, j, c):
        nonlocal best
        if best is not None and c >= best:
            return
        if i == len(s) and j == len(r):
            best = c
            return
        if i < len(s) and j < len(r):
            walk(i + 1, j + 1, c + cost(s[i], r[j]))
        if i < len(s):
            walk(i + 1, j, c + 1)
        if j < len(r):
            walk(i, j + 1, c + 1)

    walk(0, 0, 0)
    return best


def test_edit_distance_is_the_minimum_over_all_alignments():
    rng = np.random.default_rng(0)
    for _ in range(300):
        s = "".join(rng.choice(list(LET + "N"), size=int(rng.integers(0, 6))))
        r = "".join(rng.choice(list(LET + "N"), size=int(rng.integers(0, 6))))
        assert oracle.edit_distance(s, r) == _brute_distance(s, r), (s, r)


def _brute_viterbi(t, e, x):
    """Max over every state path from B = M_0 to E emitting exactly x (M and I emit)."""
    m = t.shape[0] - 1
    n = len(x)
    best = -math.inf

    def em(j, i):
        c = x[i]
        return e[j, LET.index(c)] if c in LET else 0.0

    def walk(state, j, i, score):
        nonlocal best
        # state in 0 (M), 1 (I), 2 (D) at position j, i letters emitted
        if j == m:  # E or I_m
            if i == n:
                best = max(best, score + t[m, state, 0])
            if i < n:
                walk(1, m, i + 1, score + t[m, state, 1])
            return
        if i < n:
            walk(0, j + 1, i + 1, score + t[j, state, 0] + em(j + 1, i))
            walk(1, j, i + 1, score + t[j, state, 1])
        walk(2, j + 1, i, score + t[j, state, 2])

    walk(0, 0, 0, 0.0)
    return best


def test_viterbi_is_the_best_of_all_state_paths():
    rng = np.random.default_rng(1)
    for trial in range(60):
        m = int(rng.integers(1, 4))
        train = ["".join(rng.choice(list(LET), size=max(1, m + int(rng.integers(-1, 2)))))
                 for _ in range(int(rng.integers(1, 5)))]
        _, t, e = oracle.hmm_build(train)
        for _ in range(4):
            x = "".join(rng.choice(list(LET + "N"), size=int(rng.integers(0, 5))))
            want = _brute_viterbi(t, e, x)
            got = oracle.hmm_viterbi(t, e, x)
            assert got == pytest.approx(want, abs=1e-9), (train, x)


def _all_path_scores(t, e, x):
    """The score of every state path from B = M_0 to E emitting exactly x."""
    m = t.shape[0] - 1
    n = len(x)
    out = []

    def em(j, i):
        c = x[i]
        return e[j, LET.index(c)] if c in LET else 0.0

    def walk(state, j, i, score):
        if score == -math.inf:
            return
        if j == m:
            if i == n:
                out.append(score + t[m, state, 0])
            if i < n:
                walk(1, m, i + 1, score + t[m, state, 1])
            return
        if i < n:
            walk(0, j + 1, i + 1, score + t[j, state, 0] + em(j + 1, i))
            walk(1, j, i + 1, score + t[j, state, 1])
        walk(2, j + 1, i, score + t[j, state, 2])

    walk(0, 0, 0, 0.0)
    return [v for v in out if v > -math.inf]


def test_forward_is_the_log_sum_over_all_state_paths():
    """Forward = log2 of the sum of 2^score over every path (enumerated); it is
    at least the Viterbi score and at most Viterbi + log2(number of paths)."""
    rng = np.random.default_rng(4)
    for trial in range(60):
        m = int(rng.integers(1, 4))
        train = ["".join(rng.choice(list(LET), size=max(1, m + int(rng.integers(-1, 2)))))
                 for _ in range(int(rng.integers(1, 5)))]
        _, t, e = oracle.hmm_build(train)
        for _ in range(4):
            x = "".join(rng.choice(list(LET + "N"), size=int(rng.integers(0, 5))))
            scores = _all_path_scores(t, e, x)
            top = max(scores)
            want = top + math.log2(sum(2.0 ** (v - top) for v in scores))
            got = oracle.hmm_forward(t, e, x)
            assert got == pytest.approx(want, abs=1e-9), (train, x)
            vit = oracle.hmm_viterbi(t, e, x)
            assert vit - 1e-12 <= got <= vit + math.log2(len(scores)) + 1e-12


def test_forward_of_the_empty_sequence_is_the_delete_path():
    """With no letter to emit the only path is B, D_1 .. D_m, E."""
    _, t, e = oracle.hmm_build(["ACGTA", "ACGTA", "ACTA"])
    m = t.shape[0] - 1
    want = t[0, 0, 2] + sum(t[j, 2, 2] for j in range(1, m)) + t[m, 2, 0]
    assert oracle.hmm_forward(t, e, "") == pytest.approx(want, abs=1e-12)
    assert oracle.hmm_viterbi(t, e, "") == pytest.approx(want, abs=1e-12)


def test_profile_of_identical_sequences_in_closed_form():
    R, N = "ACGTTGCA", 5
    ref, t, e = oracle.hmm_build([R] * N)
    m = len(R)
    assert ref == 0 and t.shape == (m + 1, 3, 3)
    for j in range(m):
        assert t[j, 0, 0] == pytest.approx(math.log2((N + 1) / (N + 3)))
        assert t[j, 0, 1] == pytest.approx(math.log2(1 / (N + 3)))
        assert t[j, 0, 2] == pytest.approx(math.log2(1 / (N + 3)))
        if j > 0:
            assert t[j, 1, 0] == pytest.approx(math.log2(1 / 3))  # unused states: pseudocounts only
    assert t[m, 0, 0] == pytest.approx(math.log2((N + 1) / (N + 2)))
    assert t[m, 0, 2] == -math.inf and t[0, 2, 0] == -math.inf
    for j in range(1, m + 1):
        for k, c in enumerate(LET):
            want = math.log2(4 * ((N + 1 if R[j - 1] == c else 1) / (N + 4)))
            assert e[j, k] == pytest.approx(want)
    # the reference's own score is its all-match path
    own = sum(e[j, LET.index(R[j - 1])] for j in range(1, m + 1)) + sum(t[j, 0, 0] for j in range(m + 1))
    assert oracle.hmm_viterbi(t, e, R) == pytest.approx(own)


def test_reference_is_the_most_frequent_sequence_first_on_ties():
    assert oracle.hmm_build(["AC", "GT", "GT", "AC"])[0] == 0
    assert oracle.hmm_build(["AC", "GT", "GT"])[0] == 1
    assert oracle.hmm_build(["AAA", "CCC", "GGG"])[0] == 0


def test_single_insertion_and_deletion_counts():
    R = "ACGTACGT"
    # one copy with an extra letter after column 4 and one with column 6 deleted
    ins = R[:4] + "G" + R[4:]  # the only zero-mismatch placement: after column 4
    dele = R[:5] + R[6:]
    _, t, e = oracle.hmm_build([R, R, ins, dele])
    N = 4
    # M_4 -> I_4 once (the insertion), I_4 -> M_5 once; D_6 entered once from M_5, left to M_7 once
    assert t[4, 0, 1] == pytest.approx(math.log2(2 / (N + 3)))
    assert t[4, 1, 0] == pytest.approx(math.log2(2 / 4))
    assert t[5, 0, 2] == pytest.approx(math.log2(2 / (N + 3)))
    assert t[6, 2, 0] == pytest.approx(math.log2(2 / 4))
    # scores rank the training variants above unrelated sequences
    s_ref, s_ins, s_del = (oracle.hmm_viterbi(t, e, x) for x in (R, ins, dele))
    s_far = oracle.hmm_viterbi(t, e, "TTTTTTTT")
    assert s_ref > s_ins > s_far and s_ref > s_del > s_far


def test_unknown_letters_score_as_background():
    _, t, e = oracle.hmm_build(["ACGT"] * 3)
    a = oracle.hmm_viterbi(t, e, "ACNT")
    # the N column emits log-odds 0; the best path still matches it
    want = e[1, 0] + e[2, 1] + 0.0 + e[4, 3] + sum(t[j, 0, 0] for j in range(5))
    assert a == pytest.approx(want)


def test_library_profile_builder_equals_the_oracle():
    """The library's host-side profile builder (no GPU needed) against the
    oracle's, on random training sets with repeats (reference ties), unknown
    letters, substitutions and indels: same reference, same move and emission
    scores (fp32 of the oracle's fp64)."""
    from paper_2509_13300_gb300 import ah, build, synth
    build.build()
    rng = np.random.default_rng(11)
    for trial in range(40):
        L = int(rng.integers(5, 120))
        base = "".join(rng.choice(list(LET), size=L))
        n = int(rng.integers(1, 12))
        train = []
        for _ in range(n):
            x = synth._mutate(rng, base, float(rng.uniform(0, 0.1)), float(rng.uniform(0, 0.05)))
            if rng.random() < 0.2 and x:
                i = int(rng.integers(len(x)))
                x = x[:i] + "N" + x[i + 1:]
            train.append(x if x else "A")
        if rng.random() < 0.3:
            train += [train[int(rng.integers(len(train)))]] * int(rng.integers(1, 3))  # repeats
        m, ref, t, e = ah.debug_hmm_profile(train)
        oref, T, E = oracle.hmm_build(train)
        assert (m, ref) == (T.shape[0] - 1, oref), trial
        assert np.array_equal(np.isinf(t), np.isinf(T)), trial
        fin = ~np.isinf(T)
        assert np.abs(t[fin] - T[fin]).max() <= 1e-5 and np.abs(e - E).max() <= 1e-5, trial
