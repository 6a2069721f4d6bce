"""The seeded input generators (host only): SplitMix64 against its published outputs,
counter-based draws, chunk-independent normals, and the lattice bond lists."""
import numpy as np

from paper_1307_7542_gb300 import workloads as W


def test_splitmix64_reference_outputs():
    """State 0 advanced by the golden gamma, finalised: the first outputs of the published
    generator (Steele, Lea & Flood 2014) for seed 0."""
    assert [int(v) for v in W.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_are_counter_based_and_chunk_independent():
    assert np.array_equal(W.splitmix64(7, 5, offset=11), W.splitmix64(7, 16)[11:])
    u = W.uniform(3, 10000, -1.0, 1.0)
    assert u.min() >= -1.0 and u.max() < 1.0
    a = W.normal(5, 10001)
    b = W.normal(5, 10001, chunk=37)
    assert np.array_equal(a, b) and np.all(np.isfinite(a))
    assert abs(a.mean()) < 0.05 and abs(a.std() - 1.0) < 0.05


def test_lattice_bond_lists():
    for Lx, Ly, periodic, nb in [(4, 4, True, 32), (3, 4, False, 17), (3, 6, True, 36), (2, 3, True, 9)]:
        b = W.square_bonds(Lx, Ly, periodic)
        assert b.shape == (nb, 2)
        pairs = {tuple(sorted(p)) for p in b.tolist()}
        assert len(pairs) == nb and all(i != j for i, j in pairs)
    assert W.ring_bonds(2).tolist() == [[0, 1]]
    assert len({tuple(sorted(p)) for p in W.ring_bonds(8).tolist()}) == 8
    assert W.star_bonds(7).shape == (7, 2)
