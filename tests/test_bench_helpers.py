"""Host logic of bench.py's forms (CPU): chunking a collection into whole
genomes, the rebased contig tables of a genome range, and the form workloads'
primer pairs (oligo totals 16 / 64 / 256 / 960 and the paper's four)."""
import numpy as np

import bench
import oracle
from paper_2509_13300_gb300 import countergen


def test_genome_chunks_cover_the_collection_with_whole_genomes():
    c = countergen.collection(seed=3, n_genomes=40, len_lo=1e5, len_hi=9e5)
    for cap in (1, 250_000, 2_000_000, 10**12):
        ch = bench.genome_chunks(c, cap)
        assert ch[0][0] == 0 and ch[-1][1] == 40
        assert all(a < b for a, b in ch) and all(ch[i][1] == ch[i + 1][0] for i in range(len(ch) - 1))
        goff = c.genome_off.astype(np.int64)
        for a, b in ch:  # at most cap bases, unless a single genome is longer
            assert goff[b] - goff[a] <= cap or b == a + 1


def test_sub_tables_rebase_contigs_of_a_genome_range():
    c = countergen.collection(seed=4, n_genomes=12, len_lo=1e5, len_hi=5e5)
    b0, b1, off, gen = bench.sub_tables(c, 3, 7)
    assert b0 == int(c.genome_off[3]) and b1 == int(c.genome_off[7])
    assert off[0] == 0 and int(off[-1]) == b1 - b0 and len(off) == len(gen) + 1
    assert set(gen.tolist()) == {3, 4, 5, 6}
    # the same contigs as the full table, shifted
    sel = (c.contig_genome >= 3) & (c.contig_genome < 7)
    assert np.array_equal(np.diff(off.astype(np.int64)), np.diff(c.contig_off.astype(np.int64))[sel])


def test_form_pairs():
    syn = bench.synthetic_pairs(2, (2, 3, 4, 2))
    assert [oracle.degeneracy(p["fwd"]) + oracle.degeneracy(p["rev"]) for p in syn] == [16, 64, 256, 960]
    assert [p["k"] for p in syn] == [2, 3, 4, 2]
    assert all(17 <= len(p["fwd"]) <= 25 and 17 <= len(p["rev"]) <= 25 for p in syn)
    paper = bench.paper_pairs(4)
    assert len(paper) == 4 and all(p["k"] == 4 for p in paper)
    large = bench.large_pairs()
    assert [oracle.degeneracy(p["fwd"]) + oracle.degeneracy(p["rev"]) for p in large] == [960, 64, 256]
