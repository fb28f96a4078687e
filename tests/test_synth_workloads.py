"""The timed and parity workloads follow their stated recipes, counted with plain numpy:
atom counts, fixed layers, periodicity, indenter placement and speed, the 300 K velocities,
and the number of atoms whose ACE weight is non-zero (distance to the region centre below
r_in + r_switch, minimum image in the periodic directions)."""
import numpy as np

import synth

KB = 8.617333262e-5            # eV / K
FTM = 0.0096485332             # (eV / A / amu) -> A / fs^2


def _region_counts(c):
    x = np.asarray(c["x"], dtype=np.float64)
    reg = c["region"]
    h = np.asarray(c["box"]["h"], dtype=np.float64).reshape(3, 3)
    L = np.diag(h)
    per = np.asarray(c["box"]["periodic"], dtype=bool)
    d = x - np.asarray(reg["center"])
    d[:, per] -= L[per] * np.round(d[:, per] / L[per])
    r = np.linalg.norm(d, axis=1)
    return int(np.sum(r < reg["r_in"])), int(np.sum(r < reg["r_in"] + reg["r_sw"]))


def test_w_indentation_slab_recipe():
    c = synth.configs.w_slab()
    x, v, fixed = c["x"], c["v"], c["fixed"]
    assert len(x) == 128000                                   # 40 x 40 x 40 BCC cells
    z = np.round(x[:, 2], 6)
    layers = np.unique(z)
    assert np.isclose(layers[1] - layers[0], 3.165 / 2)
    assert fixed.sum() == 4800 and np.all(z[fixed == 1] < layers[3] - 1e-6)   # bottom 3 layers
    assert tuple(c["box"]["periodic"]) == (1, 1, 0)
    assert np.allclose(np.diag(np.asarray(c["box"]["h"]).reshape(3, 3))[:2], 40 * 3.165)
    ind = c["indenter"]
    z_top = x[:, 2].max()
    assert ind["R"] == 40.0 and ind["K"] == 10.0
    assert np.isclose(ind["center"][2], z_top + 40.0 - 1.0)  # 1 A initial penetration
    assert np.allclose(c["ind_vel"], (0.0, 0.0, 1e-4))          # 10 m/s, downwards (dir -z)
    assert tuple(ind["dir"]) == (0.0, 0.0, -1.0)
    # 300 K Maxwell velocities on the free atoms, fixed atoms at rest, no net momentum
    free = fixed == 0
    assert np.all(v[~free] == 0.0)
    ke = 0.5 * c["mass"] * np.sum(v[free] ** 2) / FTM
    T = 2.0 * ke / (3.0 * free.sum() * KB)
    assert abs(T - 300.0) < 6.0, T
    assert np.abs(v[free].sum(axis=0)).max() < 1e-9 * free.sum()
    # the ACE hemisphere: r_in 50 A and a 4 A shell under the tip
    n_one, n_ace = _region_counts(c)
    assert c["region"]["r_in"] == 50.0 and c["region"]["r_sw"] == 4.0
    assert n_ace == 21241 and n_one == 16932


def test_cu_bulk_recipe():
    c = synth.configs.cu_bulk(sigma=0.0)
    assert len(c["x"]) == 2048 and tuple(c["box"]["periodic"]) == (1, 1, 1)
    n_one, n_ace = _region_counts(c)
    assert (n_one, n_ace) == (369, 767)                        # w = 1 inside 10 A, > 0 inside 13 A
    d = synth.configs.cu_bulk()
    dx = d["x"] - c["x"]
    assert abs(dx.std() - 0.05) < 0.003 and abs(dx.mean()) < 0.005   # sigma = 0.05 A displacements


def test_cu_precision_slab_recipe():
    c = synth.configs.cu_slab()
    assert len(c["x"]) == 2000000                              # 100 x 100 x 50 FCC cells
    assert c["fixed"].sum() == 3 * 2 * 100 * 100               # two atoms per cell per (001) layer
    _, n_ace = _region_counts(c)
    assert 0.045 < n_ace / len(c["x"]) < 0.055, n_ace          # the ACE hemisphere holds 5 %


def test_strained_cell_recipe():
    """Differentiation cells: BCC W, symmetric strain with entries in [-0.02, 0.02], about 1 %
    vacancies, Gaussian noise sigma = 0.1 A about the strained lattice sites."""
    for ncell, seed in ((4, 3), (8, 5), (12, 9)):
        c = synth.configs.strained_w_cell(ncell, seed)
        h = np.asarray(c["box"]["h"]).reshape(3, 3)
        F = h.T / (ncell * 3.165)                                 # h = diag(L) F^T
        e = F - np.eye(3)
        assert np.allclose(e, e.T) and np.abs(e).max() <= 0.02
        n0 = 2 * ncell ** 3
        x = np.asarray(c["x"])
        assert 0.95 * n0 <= len(x) <= n0 and tuple(c["box"]["periodic"]) == (1, 1, 1)
        if ncell >= 8:
            assert abs(1.0 - len(x) / n0 - 0.01) < 0.006            # about 1 % vacancies
        # each atom lies within noise of a strained BCC site: in half-cell units of the
        # unstrained lattice a site has three even or three odd coordinates
        s = np.linalg.solve(F, x.T).T / (3.165 / 2)
        site = np.round(s).astype(np.int64)
        par = np.mod(site, 2)
        assert np.all(par.min(axis=1) == par.max(axis=1))
        assert len(np.unique(np.mod(site, 2 * ncell), axis=0)) == len(x)   # no site twice
        noise = x - (site @ F.T) * (3.165 / 2)
        if ncell >= 8:
            assert abs(noise.std() - 0.1) < 0.01, noise.std()
