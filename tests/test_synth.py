"""The synthetic input recipe: seeded, deterministic, and with the shapes
the workloads are described with (the 8-atom H chain, the 40-atom s+p and
150-atom s+p+d lattices, the batch and serving streams, the sampled-row
density)."""
import numpy as np

from synth import (batch_molecules, h_line, lattice_molecule, serve_stream, shell_bf_offsets,
                   shell_supported_density)


def _same(a, b):
    return all(np.array_equal(getattr(a, f), getattr(b, f))
               for f in ("Z", "xyz", "shell_atom", "shell_l", "shell_nprim", "shell_prim", "exps", "coefs"))


def test_h_chain():
    m = h_line()
    assert m.natom == 8 and m.nbf == 8 and m.n_electrons == 8
    assert np.all(np.abs(m.xyz[:, 0] - 1.4 * np.arange(8)) <= 0.1)
    assert np.all(np.abs(m.xyz[:, 1:]) <= 0.1)
    assert np.all(m.shell_l == 0) and np.all(m.shell_nprim == 3)
    assert m.exps.min() >= 0.1 and m.exps.max() <= 10.0
    assert m.coefs.min() >= 0.2 and m.coefs.max() <= 1.0
    assert _same(m, h_line()) and not _same(m, h_line(seed=1))


def test_lattice_40_sp():
    m = lattice_molecule(40, 1, "sp")
    assert m.nbf == 220 and m.nshell == 140
    site = np.rint(m.xyz / 2.4)
    assert np.all(np.abs(m.xyz - 2.4 * site) <= 0.3 + 1e-12)
    assert set(np.unique(m.Z)) <= {1, 6, 8}
    for a in range(m.natom):
        ls = sorted(m.shell_l[m.shell_atom == a].tolist())
        assert ls == ([0, 0] if m.Z[a] == 1 else [0, 0, 0, 1, 1])
    assert np.all(m.shell_nprim == 3)
    assert m.exps.min() >= 0.05 and m.exps.max() <= 50.0
    assert m.n_electrons % 2 == 0 and m.Z.sum() - m.n_electrons in (0, 1)
    assert _same(m, lattice_molecule(40, 1, "sp"))


def test_lattice_150_spd():
    m = lattice_molecule(150, 2, "spd")
    assert m.nbf == 1366
    heavy = m.Z > 1
    for a in range(m.natom):
        n_d = int(np.sum((m.shell_atom == a) & (m.shell_l == 2)))
        assert n_d == (1 if heavy[a] else 0)
    assert m.shell_nprim.min() >= 1 and m.shell_nprim.max() <= 6
    assert m.exps.min() >= 0.03 and m.exps.max() <= 200.0


def test_odd_charge_sum_is_a_cation():
    for seed in range(40):
        m = lattice_molecule(5, seed, "sp")
        if m.Z.sum() % 2:
            assert m.n_electrons == m.Z.sum() - 1
            return
    raise AssertionError("no odd charge sum in 40 seeds")


def test_batch_and_serving_streams():
    mols = batch_molecules(16)
    assert all(4 <= m.natom <= 60 for m in mols)
    assert [m.seed for m in mols] == [1000 + i for i in range(16)]
    t, sizes, seeds = serve_stream(20000)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 20000 - 1 / 200.0) < 0.05 / 200.0      # mean gap 1/200 s
    assert sizes.min() >= 4 and sizes.max() <= 150
    assert np.array_equal(seeds, 10000 + np.arange(20000))
    # log-uniform sizes: the median near the geometric mean of 4 and 150
    assert abs(np.median(sizes) - np.sqrt(4 * 150)) < 3


def test_shell_supported_density():
    m = lattice_molecule(150, 2, "spd")
    D, shells, rows = shell_supported_density(m, seed=11)
    off = shell_bf_offsets(m)
    assert off[-1] == m.nbf and D.shape == (m.nbf, m.nbf)
    assert np.array_equal(D, D.T)
    assert np.linalg.eigvalsh(D).min() > -1e-12
    support = np.zeros(m.nbf, bool)
    for s in shells:
        support[off[s]:off[s + 1]] = True
    assert np.all(D[~support] == 0.0) and np.all(D[:, ~support] == 0.0)
    assert sum(m.shell_l[s] == 2 for s in shells) >= 2
    assert rows[2] == 0 and rows[3] == m.nbf // 2 and rows[4] == m.nbf - 1


def test_water_qz_shape():
    """H2O with the quadruple-zeta shape of the paper's HF benchmark: O
    5s4p3d2f1g, H 4s3p2d1f, two 12-primitive s shells and a 6-primitive p
    shell on O, a 4-primitive s shell on each H, nbf 140."""
    from synth import water_qz
    m = water_qz(0)
    assert m.natom == 3 and list(m.Z) == [8, 1, 1] and m.n_electrons == 10 and m.nbf == 140
    r = np.linalg.norm(m.xyz[1:] - m.xyz[0], axis=1)
    assert np.allclose(r, 1.809)
    v1, v2 = m.xyz[1] - m.xyz[0], m.xyz[2] - m.xyz[0]
    assert abs(np.degrees(np.arccos(v1 @ v2 / (r[0] * r[1]))) - 104.5) < 1e-9
    for atom, want in ((0, {0: 5, 1: 4, 2: 3, 3: 2, 4: 1}), (1, {0: 4, 1: 3, 2: 2, 3: 1})):
        ls = m.shell_l[m.shell_atom == atom]
        assert {l: int(np.sum(ls == l)) for l in set(ls.tolist())} == want
    on_o = m.shell_atom == 0
    assert sorted(m.shell_nprim[on_o & (m.shell_l == 0)].tolist()) == [1, 1, 1, 12, 12]
    assert sorted(m.shell_nprim[on_o & (m.shell_l == 1)].tolist()) == [1, 1, 1, 6]
    assert _same(m, water_qz(0)) and not _same(m, water_qz(1))


def test_water_cluster_qz():
    from synth import water_cluster_qz, water_qz
    w, c = water_qz(0), water_cluster_qz(8, 0)
    assert c.natom == 24 and c.nbf == 8 * w.nbf and c.n_electrons == 80
    # every copy is a rigid motion of the water: same bond lengths and basis
    for k in range(8):
        x = c.xyz[3 * k:3 * k + 3]
        assert np.allclose(np.linalg.norm(x[1:] - x[0], axis=1), 1.809)
    assert np.array_equal(c.exps, np.tile(w.exps, 8))
    d = np.linalg.norm(c.xyz[:, None] - c.xyz[None], axis=-1)
    np.fill_diagonal(d, 99.0)
    assert d.min() > 1.5
    assert _same(c, water_cluster_qz(8, 0))


def test_small_f_and_g_molecules():
    from synth import small_f_molecule, small_g_molecule
    f, g = small_f_molecule(0), small_g_molecule(0)
    assert f.shell_l.tolist() == [0, 0, 1, 3, 0, 0] and f.nbf == 17 and f.n_electrons == 8
    assert g.shell_l.tolist() == [0, 0, 1, 4, 0, 2] and g.nbf == 27 and g.n_electrons == 8
    assert f.exps.min() >= 0.3 and f.exps.max() <= 6.0
    assert _same(f, small_f_molecule(0)) and _same(g, small_g_molecule(0))


def test_spdfg_lattice_rule():
    m = lattice_molecule(3, 1, "spdfg")
    for a in range(m.natom):
        ls = sorted(m.shell_l[m.shell_atom == a].tolist())
        assert ls == ([0, 0, 1] if m.Z[a] == 1 else [0, 0, 0, 1, 1, 2, 3, 4])
