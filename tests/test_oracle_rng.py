"""Pins of the oracle's counter-based generator (Philox4x32-10) and uniforms."""
import numpy as np


def test_philox_known_answers(orc):
    # Known-answer vectors published with Philox4x32-10 (Salmon et al., SC'11,
    # Random123 distribution): counter, key -> output.
    cases = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in cases:
        assert orc.philox4x32_10(ctr, key) == want


def test_uniform_open_interval(orc):
    assert orc.uniform(0) == 0.5 / 2 ** 32
    assert orc.uniform(0xFFFFFFFF) == (2 ** 32 - 0.5) / 2 ** 32
    assert 0.0 < orc.uniform(0) < orc.uniform(1) < orc.uniform(0xFFFFFFFF) < 1.0


def test_philox_counter_words_uniform_chi2(orc):
    # every output word of consecutive counters is uniform (chi^2, 64 bins)
    n = 20000
    words = np.array([orc.philox4x32_10([i, 7, 3, 1], [0, 0]) for i in range(n)], dtype=np.uint64)
    for w in range(4):
        hist = np.bincount((words[:, w] >> np.uint64(26)).astype(np.int64), minlength=64)
        chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 63 + 5 * np.sqrt(2 * 63)


def test_six_uniforms_of_a_3d_step_use_every_bit_once(orc):
    """The 3D step's six 21-bit uniforms (reading R12) read disjoint bits of the block: a
    single set bit moves at most one of them, each takes 21 bits, and 126 of the 128 bits are
    used.  Each is (f + 1/2)/2^21 for a 21-bit integer f, on that grid inside (0, 1)."""
    base = orc.uniforms21([0, 0, 0, 0])
    assert np.all(base == 0.5 / 2 ** 21)
    hits = np.zeros(6, dtype=int)
    unused = 0
    for word in range(4):
        for bit in range(32):
            w = [0, 0, 0, 0]
            w[word] = 1 << bit
            moved = np.flatnonzero(orc.uniforms21(w) != base)
            assert len(moved) <= 1, (word, bit, moved)
            if len(moved):
                hits[moved[0]] += 1
            else:
                unused += 1
    assert list(hits) == [21] * 6 and unused == 2
    u = orc.uniforms21([0xFFFFFFFF] * 4)
    assert np.all(u == (2 ** 21 - 0.5) / 2 ** 21)


def test_six_uniforms_are_uniform_and_uncorrelated(orc):
    """Over consecutive Philox counters each of the six is uniform (chi^2, 64 bins) and the
    pairwise correlations vanish (|r| < 4 / sqrt(n))."""
    n = 20000
    u = np.array([orc.uniforms21(orc.philox4x32_10([i, 5, 2, 0], [3, 9])) for i in range(n)])
    for j in range(6):
        hist = np.bincount(np.minimum((u[:, j] * 64).astype(int), 63), minlength=64)
        chi2 = ((hist - n / 64) ** 2 / (n / 64)).sum()
        assert chi2 < 120, (j, chi2)  # 63 dof: p < 1e-5 beyond ~120
    r = np.corrcoef(u.T)
    off = r[~np.eye(6, dtype=bool)]
    assert np.all(np.abs(off) < 4 / np.sqrt(n)), off
