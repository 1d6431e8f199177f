"""Pins of the oracle's point generators (Sec. 4.1-4.3) against facts that fix them.

* Gray code order against the table printed in Sec. 4.3 (tests/golden/gray_code_b2.txt).
* Radical inverse v(i) against its digit-sum definition evaluated in floating point.
* Digital nets: every one-dimensional projection is a (0, m, 1)-net, the
  (identity, Pascal) pair is a (0, m, 2)-net, and LMS + digital shift keep both.
* Gray order is a permutation of natural order; the unshifted net is a group under XOR.
* Lattices: each coordinate is a permutation of the grid for odd g; the set is closed
  under addition mod 1; n_min..n_max sub-ranges extend the sequence (extensibility).
"""
import os
from math import comb

import numpy as np
import pytest

from oracle import qk_oracle as o
from paper_2502_14256_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gray_code_matches_printed_table():
    rows = []
    with open(os.path.join(GOLDEN, "gray_code_b2.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                i, bi, gi = ln.split()
                rows.append((int(i), int(bi, 2), int(gi, 2)))
    assert len(rows) == 9
    for i, bi, gi in rows[:8]:
        assert i == bi
        assert int(o.gray_code(np.array([i]))[0]) == gi
    # Reading: the printed b=2 code for i = 8 (1000) differs from the code for i = 7 (0100)
    # in two digits, contradicting the one-digit-change property stated beside the table;
    # the reflected code 1100 is the only one that keeps it.
    i8, _, printed8 = rows[8]
    assert bin(printed8 ^ rows[7][2]).count("1") == 2
    assert int(o.gray_code(np.array([i8]))[0]) == 0b1100
    # one digit changes per step (the property the Gray update uses)
    g = o.gray_code(np.arange(1 << 12)).astype(np.int64)
    steps = np.bitwise_xor(g[1:], g[:-1])
    assert np.all(steps & (steps - 1) == 0)


def test_radical_inverse_matches_digit_sum():
    idx = np.arange(5000, dtype=np.uint64)
    words = o.radical_inverse_word(idx).astype(np.float64) / 2 ** 32
    want = np.array([sum(((i >> (t - 1)) & 1) * 2.0 ** -t for t in range(1, 33)) for i in range(5000)])
    assert np.array_equal(words, want)
    assert np.array_equal(o.bit_reverse(np.arange(16), 4), [0, 8, 4, 12, 2, 10, 6, 14, 1, 9, 5, 13, 3, 11, 7, 15])


def _is_0m1(col_words, m):
    top = (col_words.astype(np.uint64) >> np.uint64(32 - m)).astype(np.int64)
    return np.array_equal(np.sort(top), np.arange(1 << m))


def _is_0m2(Xa, Xb, m):
    for m1 in range(m + 1):
        m2 = m - m1
        a = (Xa.astype(np.uint64) >> np.uint64(32 - m1)) if m1 else np.zeros(Xa.shape, np.uint64)
        b = (Xb.astype(np.uint64) >> np.uint64(32 - m2)) if m2 else np.zeros(Xb.shape, np.uint64)
        cells = (a << np.uint64(m2)) | b
        if not np.array_equal(np.sort(cells.astype(np.int64)), np.arange(1 << m)):
            return False
    return True


def _pascal_columns():
    return np.array([sum((comb(k, t) % 2) << (31 - t) for t in range(32)) for k in range(32)],
                    dtype=np.uint32)


@pytest.mark.parametrize("order", ["natural", "gray"])
def test_net_projections_are_0m1_nets(order):
    net = inputs.make_net(5, 6, 3, order)
    Ct = o.lms_scramble(net.C, net.S)
    for m in (1, 4, 9):
        for r in range(3):
            X = o.net_points(Ct[r], net.D[r], np.arange(1 << m), m, order)
            for j in range(6):
                assert _is_0m1(X[:, j], m), (m, r, j)


def test_pascal_pair_is_0m2_net_and_scrambling_keeps_it():
    C = np.stack([inputs.identity_columns(), _pascal_columns()])
    m = 8
    X = o.net_points(C, np.zeros(2, np.uint32), np.arange(1 << m), m, "natural")
    assert _is_0m2(X[:, 0], X[:, 1], m)
    rng = inputs.SplitMix64(99)
    S = np.stack([np.stack([inputs.random_lower_unit_rows(rng) for _ in range(2)]) for _ in range(4)])
    D = rng.u32(8).reshape(4, 2)
    Ct = o.lms_scramble(C, S)
    for r in range(4):
        for order in ("natural", "gray"):
            Xs = o.net_points(Ct[r], D[r], np.arange(1 << m), m, order)
            assert _is_0m2(Xs[:, 0], Xs[:, 1], m)
    # a deliberately bad pair (identity twice) is not a (0, m, 2)-net
    Xbad = o.net_points(np.stack([C[0], C[0]]), np.zeros(2, np.uint32), np.arange(1 << m), m, "natural")
    assert not _is_0m2(Xbad[:, 0], Xbad[:, 1], m)


def test_identity_generator_gives_van_der_corput():
    C = inputs.identity_columns()[None, :]
    X = o.net_points(C, np.zeros(1, np.uint32), np.arange(1 << 10), 10, "natural")[:, 0]
    assert np.array_equal(X.astype(np.uint64), o.radical_inverse_word(np.arange(1 << 10)))


def test_lms_identity_and_columns():
    net = inputs.make_net(3, 4, 1)
    I_rows = inputs.identity_columns()  # identity rows have the same masks as its columns
    assert np.array_equal(o.lms_scramble(net.C, I_rows[None, None, :].repeat(4, 1)), net.C[None])
    Ct = o.lms_scramble(net.C, net.S)[0]
    # point 2^k in natural order (unshifted) is exactly scrambled column k
    X = o.net_points(Ct, np.zeros(4, np.uint32), np.array([1 << k for k in range(10)]), 10, "natural")
    assert np.array_equal(X, Ct[:, :10].T)


@pytest.mark.parametrize("m", [3, 8, 11])
def test_gray_order_permutes_natural_order(m):
    net = inputs.make_net(17, 5, 2)
    Ct = o.lms_scramble(net.C, net.S)
    for r in range(2):
        Xn = o.net_points(Ct[r], net.D[r], np.arange(1 << m), m, "natural")
        Xg = o.net_points(Ct[r], net.D[r], np.arange(1 << m), m, "gray")
        assert np.array_equal(np.sort(Xn.view(np.uint32).reshape(-1, 5), axis=0), np.sort(Xg, axis=0))
        gi = o.gray_code(np.arange(1 << m)).astype(np.int64)
        assert np.array_equal(Xg, Xn[gi])


def test_unshifted_net_is_a_group_under_xor():
    net = inputs.make_net(23, 4, 1)
    Ct = o.lms_scramble(net.C, net.S)[0]
    m = 7
    Z = o.net_points(Ct, np.zeros(4, np.uint32), np.arange(1 << m), m, "natural")
    i = np.arange(1 << m)
    for k in (1, 5, 77, 127):
        assert np.array_equal(Z ^ Z[k], Z[i ^ k])


def test_lattice_coordinates_are_permutations_and_closed():
    lat = inputs.make_lattice(31, 6, 2, 10)
    m = 10
    n = 1 << m
    idx = np.arange(n)
    X0 = o.lattice_points(lat.g, np.zeros(6, np.uint32), idx)
    J = (X0.astype(np.uint64) >> np.uint64(32 - m)).astype(np.int64)
    assert np.all((X0.astype(np.uint64) & np.uint64((1 << (32 - m)) - 1)) == 0)
    for j in range(6):
        assert np.array_equal(np.sort(J[:, j]), np.arange(n))
    # z_i = i' g / n for the bit-reversed i' (linear vs natural order, Sec. 4.2)
    lin = o.bit_reverse(idx, m).astype(np.int64)
    assert np.array_equal(J, (lin[:, None] * lat.g[None, :].astype(np.int64)) % n)
    # closure: z_a + z_b mod 1 is another lattice point
    rows = {tuple(r) for r in J}
    for a, b in ((1, 2), (5, 700), (1023, 3)):
        assert tuple((J[a] + J[b]) % n) in rows
    # the shift is a mod-1 translation of every coordinate
    X = o.lattice_points(lat.g, lat.D[1], idx)
    diff = (X.astype(np.int64) - X0.astype(np.int64)) % (1 << 32)
    assert np.all(diff == lat.D[1].astype(np.int64)[None, :])


def test_sub_ranges_extend_the_sequence():
    net = inputs.make_net(41, 3, 1)
    Ct = o.lms_scramble(net.C, net.S)[0]
    full = o.net_points(Ct, net.D[0], np.arange(64), 6, "gray")
    part = o.net_points(Ct, net.D[0], np.arange(16, 64), 6, "gray")
    assert np.array_equal(full[16:], part)
    # a larger m reproduces the first 2^m points (natural and Gray order are extensible)
    big = o.net_points(Ct, net.D[0], np.arange(64), 12, "gray")
    assert np.array_equal(full, big)
    lat = inputs.make_lattice(43, 3, 1, 12)
    assert np.array_equal(o.lattice_points(lat.g, lat.D[0], np.arange(8, 32)),
                          o.lattice_points(lat.g, lat.D[0], np.arange(32))[8:])


def test_digital_shift_is_a_xor_of_every_point():
    net = inputs.make_net(61, 5, 2)
    Ct = o.lms_scramble(net.C, net.S)[1]
    idx = np.arange(300)
    Z = o.net_points(Ct, np.zeros(5, np.uint32), idx, 9)
    X = o.net_points(Ct, net.D[1], idx, 9)
    assert np.all((X ^ Z) == net.D[1][None, :])
    assert np.any(net.D[1] != 0)


def test_splitmix64_known_answers_and_chunking():
    """The seeded input generator is SplitMix64 (Steele, Lea & Flood 2014): its first outputs
    for seed 1234567 are the widely published test vector of the generator's reference C
    code, and drawing in chunks continues the same stream."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    assert [int(v) for v in inputs.SplitMix64(1234567).next_u64(5)] == want
    a = inputs.SplitMix64(42).next_u64(10)
    g = inputs.SplitMix64(42)
    b = np.concatenate([g.next_u64(3), g.next_u64(0), g.next_u64(7)])
    assert np.array_equal(a, b)
