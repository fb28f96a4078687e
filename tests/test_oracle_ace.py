"""Pins of the oracle's synthetic ACE (Sec. 2.2.2, Eq. energy_ace).

The product basis is checked against brute-force sums over neighbour pairs and triples
that never touch Y_lm or the Gaunt table: by the addition theorem,
  sum_m A_n1lm A_n2lm          = nref^-2 sum_jk g g (2l+1)/(4 pi) P_l(rhat_j . rhat_k),
  sum_m G A_n1l1m1 A_.. A_..   = nref^-3 int dOmega_s prod_a [sum_j g (2l_a+1)/(4 pi) P_la(rhat_j . s)],
with numpy's Chebyshev series and scipy's Legendre polynomials.  Special cases reduce
the energy to a pair potential and to a Finnis-Sinclair square root.
"""
import numpy as np
import pytest
from scipy.special import eval_legendre

import synth

rng = np.random.default_rng(7)


def _nbrs(n=9, rmin=2.2, rmax=4.9):
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * rng.uniform(rmin, rmax, size=(n, 1))


def _g(r, rc, n):
    c = np.zeros(n + 1); c[n] = 1
    return np.where(r < rc, np.polynomial.chebyshev.chebval(2 * r / rc - 1, c) * 0.5 * (1 + np.cos(np.pi * r / rc)), 0.0)


def _sphere_quadrature(nt=12, nphi=26):
    xs, ws = np.polynomial.legendre.leggauss(nt)
    S, W = [], []
    for ct, wt in zip(xs, ws):
        st = np.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * np.pi * k / nphi
            S.append([st * np.cos(ph), st * np.sin(ph), ct]); W.append(wt * 2 * np.pi / nphi)
    return np.array(S), np.array(W)


def test_basis_list_is_the_stated_one():
    idx = synth.ace_basis(8, 4)
    nu = idx[:, 0]
    assert (nu == 1).sum() == 8 and (nu == 2).sum() == 180 and (nu == 3).sum() == 3976
    t = idx[nu == 3]
    assert np.all((t[:, 2] + t[:, 4] + t[:, 6]) % 2 == 0)
    assert np.all(np.abs(t[:, 2] - t[:, 4]) <= t[:, 6]) and np.all(t[:, 6] <= t[:, 2] + t[:, 4])
    keys = [tuple(r) for r in t[:, 1:]]
    assert len(set(keys)) == len(keys)


def test_product_basis_against_brute_force(orc):
    ace = synth.ace_potential("W")
    rv = _nbrs()
    out = orc.ace_atom(ace, rv)
    B = out["B"]
    r = np.linalg.norm(rv, axis=1)
    u = rv / r[:, None]
    nref, rc = ace["nref"], ace["rc"]
    g = np.array([_g(r, rc, n) for n in range(8)])            # (n, j)
    idx = ace["idx"]
    # nu = 1
    for v in np.where(idx[:, 0] == 1)[0]:
        assert abs(B[v] - g[idx[v, 1]].sum() / np.sqrt(4 * np.pi) / nref) < 1e-13
    # nu = 2
    cos = u @ u.T
    for v in np.where(idx[:, 0] == 2)[0]:
        _, n1, l, n2, _, _, _ = idx[v]
        ref = np.einsum("j,k,jk->", g[n1], g[n2], (2 * l + 1) / (4 * np.pi) * eval_legendre(l, cos)) / nref ** 2
        assert abs(B[v] - ref) < 1e-12
    # nu = 3 (a sample of 300 functions)
    S, W = _sphere_quadrature()
    cs = u @ S.T                                               # (j, s)
    P = {l: (2 * l + 1) / (4 * np.pi) * eval_legendre(l, cs) for l in range(5)}
    v3 = np.where(idx[:, 0] == 3)[0]
    for v in rng.choice(v3, size=300, replace=False):
        _, n1, l1, n2, l2, n3, l3 = idx[v]
        f1, f2, f3 = g[n1] @ P[l1], g[n2] @ P[l2], g[n3] @ P[l3]   # functions of s
        ref = np.sum(W * f1 * f2 * f3) / nref ** 3
        assert abs(B[v] - ref) < 1e-12 * max(1.0, abs(ref)), (idx[v], B[v], ref)


def test_every_basis_function_is_rotation_invariant(orc):
    ace = synth.ace_potential("Cu")
    rv = _nbrs(12)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    a = orc.ace_atom(ace, rv)
    b = orc.ace_atom(ace, rv @ q.T)
    c = orc.ace_atom(ace, rv[rng.permutation(len(rv))])
    assert np.abs(a["B"] - b["B"]).max() < 1e-12
    assert np.abs(a["B"] - c["B"]).max() < 1e-12
    assert abs(a["E"] - b["E"]) < 1e-12
    # forces rotate with the frame
    assert np.abs(a["f"] @ q.T - b["f"]).max() < 1e-11


def test_ace_pair_forces_are_the_energy_gradient(orc):
    ace = synth.ace_potential("W")
    rv = _nbrs(10)
    out = orc.ace_atom(ace, rv)
    h = 1e-5
    for j in range(len(rv)):
        for k in range(3):
            p = rv.copy(); p[j, k] += h
            m = rv.copy(); m[j, k] -= h
            fd = (orc.ace_atom(ace, p)["E"] - orc.ace_atom(ace, m)["E"]) / (2 * h)
            assert abs(fd - out["f"][j, k]) < 1e-8


def test_linear_nu1_reduces_to_a_pair_potential(orc):
    ace = synth.ace_potential("Cu")
    nu1 = ace["idx"][:, 0] == 1
    ace["c1"] = np.where(nu1, ace["c1"], 0.0)
    ace["c2"] = np.zeros_like(ace["c2"])
    rv = _nbrs(11)
    r = np.linalg.norm(rv, axis=1)
    ref = ace["c1_0"] + np.sqrt(ace["c2_0"]) + sum(
        ace["c1"][v] * _g(r, ace["rc"], ace["idx"][v, 1]).sum() for v in np.where(nu1)[0]) / np.sqrt(4 * np.pi) / ace["nref"]
    assert abs(orc.ace_atom(ace, rv)["E"] - ref) < 1e-13


def test_sqrt_nu1_reduces_to_finnis_sinclair(orc):
    ace = synth.ace_potential("W")
    nu1 = ace["idx"][:, 0] == 1
    ace["c1"] = np.zeros_like(ace["c1"])
    ace["c1_0"] = 0.0
    ace["c2"] = np.where(nu1, np.abs(ace["c2"]), 0.0)
    rv = _nbrs(8)
    r = np.linalg.norm(rv, axis=1)
    dens = sum(ace["c2"][v] * _g(r, ace["rc"], ace["idx"][v, 1]).sum() for v in np.where(nu1)[0]) / np.sqrt(4 * np.pi) / ace["nref"]
    assert abs(orc.ace_atom(ace, rv)["E"] - np.sqrt(ace["c2_0"] + dens)) < 1e-13


def test_isolated_atom_and_domain_error(orc):
    ace = synth.ace_potential("W")
    out = orc.ace_atom(ace, np.zeros((0, 3)))
    assert out["status"] == 0 and abs(out["E"] - (ace["c1_0"] + np.sqrt(ace["c2_0"]))) < 1e-14
    ace["c2_0"] = -1.0
    assert orc.ace_atom(ace, _nbrs(4))["status"] == -4


@pytest.mark.parametrize("species", ["Cu", "W"])
def test_phi2_stays_positive_on_the_workloads(orc, species):
    c = synth.configs.cu_bulk() if species == "Cu" else synth.configs.w_bulk()
    pi, pj, rv = orc.neighbors(c["x"], c["box"], c["ace"]["rc"])
    for i in range(0, len(c["x"]), 37):
        o = orc.ace_atom(c["ace"], rv[pi == i])
        assert o["phi2"] > 1.0
