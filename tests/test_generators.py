"""The counter-based input generator (large and served workloads): Philox4x32-10
against the published known-answer vectors, and chunk independence of the
collection bases (any range is a function of its positions alone)."""
import numpy as np

from paper_2509_13300_gb300 import countergen


def test_philox_known_answer_vectors():
    """Philox4x32-10 known-answer vectors (Salmon et al., SC 2011; the Random123
    distribution's test vectors): zero counter and key, all-ones, and the pi digits."""
    ctr = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]], dtype=np.uint32)
    keys = [(0, 0), (0xFFFFFFFF, 0xFFFFFFFF), (0xA4093822, 0x299F31D0)]
    want = [[0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8], [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD],
            [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]]
    for c, k, w in zip(ctr, keys, want):
        assert countergen.philox4x32(c[None, :], k)[0].tolist() == w


def test_collection_bases_are_chunk_independent():
    c = countergen.collection(seed=11, n_genomes=4, len_lo=5e4, len_hi=2e5)
    full = c.bases()
    assert len(full) == c.n_bases
    cuts = [0, 4, 1000, 12345, 77777, c.n_bases]
    parts = np.concatenate([c.bases(a, b) for a, b in zip(cuts[:-1], cuts[1:])])
    assert np.array_equal(parts, full)
    # composition follows the thresholds: no letter outside ACGTN, N only in N segments
    assert set(np.unique(full).tolist()) <= set(b"ACGTN")
    n_seg = c.segments[c.segments["letter"] != 0]
    n_total = int(np.sum(np.diff(np.concatenate([[0], c.segments["end"]]))[c.segments["letter"] != 0]))
    assert int((full == ord("N")).sum()) <= n_total and len(n_seg) > 0
    # the planted patches are present
    assert np.array_equal(full[c.patch_pos.astype(np.int64)], c.patch_bytes)


def test_collection_layout_invariants():
    """The vectorised layout: genome lengths in range, contigs inside their
    genomes and in order, segments tiling the collection, about 0.1 % N."""
    c = countergen.collection(seed=7, n_genomes=300, len_lo=1e5, len_hi=8e5)
    goff = c.genome_off.astype(np.int64)
    lens = np.diff(goff)
    assert goff[0] == 0 and goff[-1] == c.n_bases
    assert lens.min() >= 1e5 - 1 and lens.max() <= 8e5 + 1
    coff = c.contig_off.astype(np.int64)
    assert np.all(np.diff(coff) >= 0) and coff[0] == 0 and coff[-1] == c.n_bases
    owner = np.searchsorted(goff, coff[:-1], side="right") - 1
    assert np.array_equal(owner, c.contig_genome)
    assert np.all(np.diff(c.contig_genome.astype(np.int64)) >= 0)
    ends = c.segments["end"].astype(np.int64)
    assert np.all(np.diff(ends) >= 0) and ends[-1] == c.n_bases
    seg_len = np.diff(np.concatenate([[0], ends]))
    n_frac = seg_len[c.segments["letter"] != 0].sum() / c.n_bases
    assert 0.0005 < n_frac < 0.0015
    # patches lie inside the collection, sorted and unique
    pp = c.patch_pos.astype(np.int64)
    assert len(pp) > 0 and np.all(np.diff(pp) > 0) and pp[-1] < c.n_bases


def test_operon_family_plants_homologous_amplicons():
    from paper_2509_13300_gb300 import synth
    w = synth.operon_family(seed=5, n_genomes=4, genome_len=60_000, template_len=400)
    assert len(w.contig_genome) == 4 and w.n_bases == 240_000
    p = w.pairs[0]
    assert len(p["fwd"]) == 20 and len(p["rev"]) == 20 and p["max_len"] == 800


def test_encode_2bit_round_trip():
    """The 2-bit host encoding of ah_load_genomes_2bit: decoding the codes and
    the no-base runs gives the input upper-cased, every non-ACGT letter as N."""
    from paper_2509_13300_gb300 import ah
    rng = np.random.default_rng(4)
    letters = np.frombuffer(b"ACGTacgtNnRYKM-.", dtype=np.uint8)
    for n in (0, 1, 3, 4, 5, 1000, 4097):
        seq = letters[rng.integers(0, len(letters), n)] if n else np.zeros(0, np.uint8)
        codes, gaps = ah.encode_2bit(seq)
        assert len(codes) == (n + 3) // 4 and gaps.shape[1] == 2
        dec = np.array([b"ACGT"[(codes[p // 4] >> (2 * (p % 4))) & 3] for p in range(n)], dtype=np.uint8)
        for a, ln in gaps.tolist():
            dec[a:a + ln] = ord("N")
        want = np.array([ch - 32 if 97 <= ch <= 122 else ch for ch in seq.tolist()], dtype=np.uint8)
        want = np.where(np.isin(want, np.frombuffer(b"ACGT", np.uint8)), want, ord("N")).astype(np.uint8)
        assert dec.tobytes() == want.tobytes()
        # runs are sorted, disjoint, non-empty and maximal
        if len(gaps) > 1:
            assert np.all(gaps[1:, 0] > gaps[:-1, 0] + gaps[:-1, 1])
        assert np.all(gaps[:, 1] >= 1) if len(gaps) else True
