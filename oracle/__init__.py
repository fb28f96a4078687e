"""Python wrapper of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference legs may import this package.  It shares no code with the
CUDA library (paper_2505_12958_gb300) and does not import it.

Each function cites the passage of arXiv 2505.12958 it follows in oracle.c.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

D = C.c_double
I = C.c_int
PD = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)
PU8 = C.POINTER(C.c_ubyte)


def build(force=False):
    """Compile oracle.c with gcc (IEEE double, no fast-math; OpenMP over atoms)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-D_DEFAULT_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class EAM(C.Structure):
    _fields_ = [("n_phi", I), ("phi_a", D * 32), ("phi_d", D * 32),
                ("n_rho", I), ("rho_a", D * 16), ("rho_d", D * 16), ("rho_rclamp", D),
                ("F_a1", D), ("F_a2", D), ("F_dxi", D),
                ("zbl", I), ("zbl_Z", D), ("zbl_eps0", D), ("zbl_a", D), ("r_lo", D), ("r_hi", D),
                ("b", D * 6)]


class ACE(C.Structure):
    _fields_ = [("rc", D), ("nref", D), ("nmax", I), ("lmax", I), ("nfunc", I),
                ("idx", PI), ("c1", PD), ("c2", PD), ("c1_0", D), ("c2_0", D)]


class System(C.Structure):
    _fields_ = [("n", I), ("x", PD), ("h", D * 9), ("origin", D * 3), ("periodic", I * 3)]


class Region(C.Structure):
    _fields_ = [("kind", I), ("center", D * 3), ("r_in", D), ("r_sw", D),
                ("w_explicit", PD), ("w_const", D)]


class Indenter(C.Structure):
    _fields_ = [("enabled", I), ("center", D * 3), ("R", D), ("K", D), ("dir", D * 3)]


class Result(C.Structure):
    _fields_ = [("e_total", D), ("virial", D * 6), ("load", D), ("e_indenter", D),
                ("n_ace", I), ("status", I), ("bad_atom", I)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_evaluate.restype = I
        L.or_evaluate.argtypes = [C.POINTER(System), C.POINTER(EAM), C.POINTER(ACE), C.POINTER(Region),
                                  C.POINTER(Indenter), PU8, I, PD, PD, PD, PD, PD, C.POINTER(Result)]
        L.or_neighbors.restype = C.c_long
        L.or_neighbors.argtypes = [C.POINTER(System), D, I, C.c_long, PI, PI, PD]
        for fn in ("or_eam_phi", "or_eam_rho", "or_eam_embed"):
            getattr(L, fn).restype = None
            getattr(L, fn).argtypes = [C.POINTER(EAM), D, PD, PD]
        L.or_eam_cutoff.restype = D
        L.or_eam_cutoff.argtypes = [C.POINTER(EAM)]
        L.or_ylm.restype = None
        L.or_ylm.argtypes = [D, D, D, PD, PD]
        L.or_radial.restype = None
        L.or_radial.argtypes = [D, D, I, PD, PD]
        L.or_gaunt.restype = D
        L.or_gaunt.argtypes = [I, I, I, I, I, I]
        L.or_ace_atom.restype = I
        L.or_ace_atom.argtypes = [C.POINTER(ACE), I, PD, PD, PD, PD, PD, PD]
        L.or_md.restype = I
        L.or_md.argtypes = [C.POINTER(System), C.POINTER(EAM), C.POINTER(ACE), C.POINTER(Region),
                            C.POINTER(Indenter), PD, I, PU8, D, D, I, I, PD, PD, PD, PD]
        L.or_num_threads.restype = I
        L.or_md_nh.restype = I
        L.or_md_nh.argtypes = [C.POINTER(System), C.POINTER(EAM), C.POINTER(ACE), C.POINTER(Region),
                               C.POINTER(Indenter), PD, I, PU8, PU8, D, D, D, D, I, I, PD, PD, PD, PD, PD]
        L.or_philox4x32_10.restype = None
        L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint), C.POINTER(C.c_uint), C.POINTER(C.c_uint)]
        L.or_md_langevin.restype = I
        L.or_md_langevin.argtypes = [C.POINTER(System), C.POINTER(EAM), C.POINTER(ACE), C.POINTER(Region),
                                     C.POINTER(Indenter), PD, I, PU8, PU8, D, D, C.c_ulonglong, I, D, D, I, I,
                                     PD, PD, PD, PD]
        L.or_csp.restype = I
        L.or_csp.argtypes = [C.POINTER(System), I, D, PD, PI]
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(PD)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_eam(p):
    if p is None:
        return None
    e = EAM()
    e.n_phi = len(p["phi_a"])
    e.n_rho = len(p["rho_a"])
    for k in range(e.n_phi):
        e.phi_a[k] = float(p["phi_a"][k]); e.phi_d[k] = float(p["phi_d"][k])
    for k in range(e.n_rho):
        e.rho_a[k] = float(p["rho_a"][k]); e.rho_d[k] = float(p["rho_d"][k])
    e.rho_rclamp = float(p.get("rho_rclamp", 0.0))
    e.F_a1, e.F_a2, e.F_dxi = float(p["F_a1"]), float(p["F_a2"]), float(p.get("F_dxi", 0.0))
    e.zbl = int(p.get("zbl", 0))
    if e.zbl:
        e.zbl_Z, e.zbl_eps0, e.zbl_a = float(p["zbl_Z"]), float(p["zbl_eps0"]), float(p["zbl_a"])
        e.r_lo, e.r_hi = float(p["r_lo"]), float(p["r_hi"])
        for k in range(6):
            e.b[k] = float(p["b"][k])
    return e


class _AceHolder:
    """Keeps the numpy arrays behind an ACE struct alive."""

    def __init__(self, p):
        self.idx = np.ascontiguousarray(p["idx"], dtype=np.int32).ravel()
        self.c1 = _f64(p["c1"])
        self.c2 = _f64(p["c2"])
        s = ACE()
        s.rc, s.nref = float(p["rc"]), float(p["nref"])
        s.nmax, s.lmax = int(p["nmax"]), int(p["lmax"])
        s.nfunc = len(self.c1)
        s.idx = self.idx.ctypes.data_as(PI)
        s.c1, s.c2 = _pd(self.c1), _pd(self.c2)
        s.c1_0, s.c2_0 = float(p["c1_0"]), float(p["c2_0"])
        self.s = s


def make_ace(p):
    return None if p is None else _AceHolder(p)


def make_system(x, box):
    x = _f64(x).reshape(-1, 3)
    s = System()
    s.n = x.shape[0]
    s.x = _pd(x)
    h = np.asarray(box["h"], dtype=np.float64).ravel()
    for k in range(9):
        s.h[k] = h[k]
    for k in range(3):
        s.origin[k] = float(box.get("origin", (0, 0, 0))[k])
        s.periodic[k] = int(box["periodic"][k])
    return s, x


def make_region(reg, n=None):
    """reg: None (w = 0), {'kind': 'sphere', center, r_in, r_sw}, {'kind': 'explicit', 'w': array},
    or {'kind': 'const', 'w': value}."""
    if reg is None:
        return None, None
    r = Region()
    keep = None
    if reg["kind"] == "sphere":
        r.kind = 1
        for k in range(3):
            r.center[k] = float(reg["center"][k])
        r.r_in, r.r_sw = float(reg["r_in"]), float(reg["r_sw"])
    elif reg["kind"] == "explicit":
        r.kind = 0
        keep = _f64(reg["w"])
        r.w_explicit = _pd(keep)
    elif reg["kind"] == "const":
        r.kind = 2
        r.w_const = float(reg["w"])
    else:
        raise ValueError(reg["kind"])
    return r, keep


def make_indenter(ind):
    if ind is None:
        return None
    s = Indenter()
    s.enabled = 1
    for k in range(3):
        s.center[k] = float(ind["center"][k])
        s.dir[k] = float(ind.get("dir", (0.0, 0.0, -1.0))[k])
    s.R, s.K = float(ind["R"]), float(ind["K"])
    return s


def _ptr(s, T):
    return C.byref(s) if s is not None else C.POINTER(T)()


def evaluate(x, box, eam=None, ace=None, region=None, indenter=None, centers=None, nthreads=0):
    """AP energy and forces (Eq. energy_hyb with w = 1 - lambda; Eqs. energy_eam, energy_ace,
    V_indenter, P_ind).  Returns a dict of numpy arrays and scalars."""
    L = lib()
    sysd, xk = make_system(x, box)
    n = sysd.n
    e = make_eam(eam)
    a = make_ace(ace)
    r, rkeep = make_region(region)
    ind = make_indenter(indenter)
    cmask = None
    if centers is not None:
        cmask = np.zeros(n, dtype=np.uint8)
        cmask[np.asarray(centers)] = 1
    F = np.zeros((n, 3))
    ea, ee, eace, w = np.zeros(n), np.zeros(n), np.zeros(n), np.zeros(n)
    res = Result()
    L.or_evaluate(C.byref(sysd), _ptr(e, EAM), C.byref(a.s) if a else C.POINTER(ACE)(),
                  _ptr(r, Region), _ptr(ind, Indenter),
                  cmask.ctypes.data_as(PU8) if cmask is not None else PU8(), int(nthreads),
                  _pd(F), _pd(ea), _pd(ee), _pd(eace), _pd(w), C.byref(res))
    del xk, rkeep
    return {"forces": F, "e_atom": ea, "e_eam": ee, "e_ace": eace, "w": w,
            "e_total": res.e_total, "virial": np.array(res.virial[:]), "load": res.load,
            "e_indenter": res.e_indenter, "n_ace": res.n_ace, "status": res.status,
            "bad_atom": res.bad_atom}


def neighbors(x, box, rc, mode=0):
    """All (i, j, r_j(image) - r_i) with |r| < rc; mode 0 cell list, 1 brute force."""
    L = lib()
    sysd, xk = make_system(x, box)
    cap = max(1024, int(sysd.n) * 256)
    while True:
        pi = np.zeros(cap, dtype=np.int32)
        pj = np.zeros(cap, dtype=np.int32)
        rv = np.zeros((cap, 3))
        cnt = L.or_neighbors(C.byref(sysd), float(rc), int(mode), cap,
                             pi.ctypes.data_as(PI), pj.ctypes.data_as(PI), _pd(rv))
        if cnt >= 0:
            return pi[:cnt], pj[:cnt], rv[:cnt]
        cap *= 4


def eam_funcs(eam, r):
    """(Phi, Phi', zeta, zeta') at the distances r (Appendix B forms)."""
    L = lib()
    e = make_eam(eam)
    out = np.zeros((len(r), 4))
    f, df = D(), D()
    for k, rr in enumerate(np.asarray(r, dtype=np.float64)):
        L.or_eam_phi(C.byref(e), rr, C.byref(f), C.byref(df)); out[k, 0], out[k, 1] = f.value, df.value
        L.or_eam_rho(C.byref(e), rr, C.byref(f), C.byref(df)); out[k, 2], out[k, 3] = f.value, df.value
    return out


def eam_embed(eam, rho):
    L = lib()
    e = make_eam(eam)
    f, df = D(), D()
    L.or_eam_embed(C.byref(e), float(rho), C.byref(f), C.byref(df))
    return f.value, df.value


def ylm(v):
    """Real orthonormal Y_lm (l <= 4) at direction v and the gradient with respect to v."""
    L = lib()
    Y = np.zeros(25)
    G = np.zeros(75)
    L.or_ylm(float(v[0]), float(v[1]), float(v[2]), _pd(Y), _pd(G))
    return Y, G.reshape(25, 3)


def radial(r, rc, nmax=8):
    L = lib()
    g, dg = np.zeros(nmax), np.zeros(nmax)
    L.or_radial(float(r), float(rc), int(nmax), _pd(g), _pd(dg))
    return g, dg


def gaunt(l1, m1, l2, m2, l3, m3):
    return lib().or_gaunt(l1, m1, l2, m2, l3, m3)


def ace_atom(ace, rvec):
    """One ACE atom (Eq. energy_ace): E, phi1, phi2, all B_v, and dE/dr_ij per neighbour."""
    L = lib()
    a = make_ace(ace)
    rv = _f64(rvec).reshape(-1, 3)
    nn = rv.shape[0]
    E, p1, p2 = D(), D(), D()
    B = np.zeros(a.s.nfunc)
    f = np.zeros((max(nn, 1), 3))
    st = L.or_ace_atom(C.byref(a.s), nn, _pd(rv), C.byref(E), C.byref(p1), C.byref(p2), _pd(B), _pd(f))
    return {"E": E.value, "phi1": p1.value, "phi2": p2.value, "B": B, "f": f[:nn], "status": st}


def md(x, v, box, eam, ace, region, indenter, ind_vel, fixed, mass, dt, nsteps,
       region_follows=False, nthreads=0):
    """Velocity Verlet.  Returns (x, v, epot[nsteps+1], ekin[nsteps+1], status)."""
    L = lib()
    x = _f64(x).reshape(-1, 3).copy()
    v = _f64(v).reshape(-1, 3).copy()
    sysd, _ = make_system(x, box)
    sysd.x = _pd(x)
    e = make_eam(eam)
    a = make_ace(ace)
    r, rkeep = make_region(region)
    ind = make_indenter(indenter)
    iv = _f64(ind_vel if ind_vel is not None else np.zeros(3))
    fx = np.ascontiguousarray(fixed, dtype=np.uint8) if fixed is not None else None
    ep, ek = np.zeros(nsteps + 1), np.zeros(nsteps + 1)
    st = L.or_md(C.byref(sysd), _ptr(e, EAM), C.byref(a.s) if a else C.POINTER(ACE)(), _ptr(r, Region),
                 _ptr(ind, Indenter), _pd(iv), int(region_follows),
                 fx.ctypes.data_as(PU8) if fx is not None else PU8(), float(mass), float(dt),
                 int(nsteps), int(nthreads), _pd(x), _pd(v), _pd(ep), _pd(ek))
    del rkeep
    return x, v, ep, ek, st


def md_nh(x, v, box, eam, ace, region, indenter, ind_vel, fixed, group, t_target, tau, mass, dt, nsteps,
          region_follows=False, nthreads=0):
    """Velocity Verlet with a Nose-Hoover thermostat on `group` (or_md_nh).  Returns
    (x, v, epot[nsteps+1], ekin[nsteps+1], ethermo[nsteps+1], status)."""
    L = lib()
    x = _f64(x).reshape(-1, 3).copy()
    v = _f64(v).reshape(-1, 3).copy()
    sysd, _ = make_system(x, box)
    sysd.x = _pd(x)
    e = make_eam(eam)
    a = make_ace(ace)
    r, rkeep = make_region(region)
    ind = make_indenter(indenter)
    iv = _f64(ind_vel if ind_vel is not None else np.zeros(3))
    fx = np.ascontiguousarray(fixed, dtype=np.uint8) if fixed is not None else None
    gr = np.ascontiguousarray(group, dtype=np.uint8)
    ep, ek, et = np.zeros(nsteps + 1), np.zeros(nsteps + 1), np.zeros(nsteps + 1)
    st = L.or_md_nh(C.byref(sysd), _ptr(e, EAM), C.byref(a.s) if a else C.POINTER(ACE)(), _ptr(r, Region),
                    _ptr(ind, Indenter), _pd(iv), int(region_follows),
                    fx.ctypes.data_as(PU8) if fx is not None else PU8(), gr.ctypes.data_as(PU8),
                    float(t_target), float(tau), float(mass), float(dt), int(nsteps), int(nthreads),
                    _pd(x), _pd(v), _pd(ep), _pd(ek), _pd(et))
    del rkeep
    return x, v, ep, ek, et, st


def philox4x32_10(ctr, key):
    """The four 32-bit words of Philox4x32-10 at counter ctr (4 words) and key (2 words)."""
    L = lib()
    c = (C.c_uint * 4)(*[int(v) & 0xffffffff for v in ctr])
    k = (C.c_uint * 2)(*[int(v) & 0xffffffff for v in key])
    o = (C.c_uint * 4)()
    L.or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def md_langevin(x, v, box, eam, ace, region, indenter, ind_vel, fixed, group, t_target, tau, seed, zero_every,
                mass, dt, nsteps, region_follows=False, nthreads=0):
    """Velocity Verlet with a Langevin thermostat on `group` (or_md_langevin).  Returns
    (x, v, epot[nsteps+1], ekin[nsteps+1], status)."""
    L = lib()
    x = _f64(x).reshape(-1, 3).copy()
    v = _f64(v).reshape(-1, 3).copy()
    sysd, _ = make_system(x, box)
    sysd.x = _pd(x)
    e = make_eam(eam)
    a = make_ace(ace)
    r, rkeep = make_region(region)
    ind = make_indenter(indenter)
    iv = _f64(ind_vel if ind_vel is not None else np.zeros(3))
    fx = np.ascontiguousarray(fixed, dtype=np.uint8) if fixed is not None else None
    gr = np.ascontiguousarray(group, dtype=np.uint8)
    ep, ek = np.zeros(nsteps + 1), np.zeros(nsteps + 1)
    st = L.or_md_langevin(C.byref(sysd), _ptr(e, EAM), C.byref(a.s) if a else C.POINTER(ACE)(), _ptr(r, Region),
                          _ptr(ind, Indenter), _pd(iv), int(region_follows),
                          fx.ctypes.data_as(PU8) if fx is not None else PU8(), gr.ctypes.data_as(PU8),
                          float(t_target), float(tau), int(seed), int(zero_every), float(mass), float(dt),
                          int(nsteps), int(nthreads), _pd(x), _pd(v), _pd(ep), _pd(ek))
    del rkeep
    return x, v, ep, ek, st


def csp(x, box, n_nb, rc):
    """Centro-symmetry parameter per atom (or_csp): the sum of the n_nb/2 smallest
    |R_j + R_k|^2 over pairs of the n_nb nearest neighbours within rc; -1 for atoms with
    fewer than n_nb neighbours there.  Returns (csp, coordination within rc)."""
    L = lib()
    sysd, xk = make_system(x, box)
    n = sysd.n
    out = np.zeros(n)
    coord = np.zeros(n, dtype=np.int32)
    st = L.or_csp(C.byref(sysd), int(n_nb), float(rc), _pd(out), coord.ctypes.data_as(PI))
    del xk
    if st != 0:
        raise ValueError("or_csp: bad arguments")
    return out, coord


def csp_weights(x, box, csp_blocks, p, w_old):
    """CSP-driven switching weights (the switching function of Appendix B, Sec. 2.2.3), the
    library's stated reading written out with numpy:
      block average of the CSP evaluations of each atom (csp_blocks: list of per-atom CSP
      arrays, -1 = surface); an atom is a surface atom when more than half of them are -1
      (or all); w0 = clamp((avg - csp_lo)/(csp_hi - csp_lo), 0, 1); w0 = 1 inside the zone
      |r - zone_center| < zone_r (nearest image); w0 = 0 for surface atoms outside it;
      w_i = max_j w0_j T(|r_ij|) over all j (itself included) and every periodic image,
      T = 1 for r <= r_lo, cos^2(pi (r - r_lo) / (2 (r_hi - r_lo))) below r_hi, else 0;
      w_i keeps its old value unless |w_new - w_old| >= dlam_min.
    Returns (w, w0)."""
    x = _f64(x).reshape(-1, 3)
    n = len(x)
    blocks = np.asarray(csp_blocks, dtype=np.float64).reshape(-1, n)
    under = (blocks < 0).sum(axis=0)
    nacc = blocks.shape[0]
    with np.errstate(invalid="ignore", divide="ignore"):
        avg = np.where(blocks < 0, 0.0, blocks).sum(axis=0) / (nacc - under)
    t = (avg - p["csp_lo"]) / (p["csp_hi"] - p["csp_lo"])
    w0 = np.clip(np.nan_to_num(t, nan=0.0), 0.0, 1.0)
    surface = (2 * under > nacc) | (under == nacc)
    w0[surface] = 0.0
    h = np.asarray(box["h"], dtype=np.float64).reshape(3, 3)
    d = x - np.asarray(p["zone_center"], dtype=np.float64)
    s = d @ np.linalg.inv(h)
    for k in range(3):
        if box["periodic"][k]:
            s[:, k] -= np.floor(s[:, k] + 0.5)
    d = s @ h
    zone = (d * d).sum(axis=1) < p["zone_r"] ** 2
    w0[zone] = 1.0
    w = w0.copy()
    pi, pj, rv = neighbors(x, box, p["r_hi"])
    r = np.sqrt((rv * rv).sum(axis=1))
    T = np.where(r <= p["r_lo"], 1.0, np.cos(0.5 * np.pi * (r - p["r_lo"]) / (p["r_hi"] - p["r_lo"])) ** 2)
    T[r >= p["r_hi"]] = 0.0
    np.maximum.at(w, pi, w0[pj] * T)
    w_old = np.asarray(w_old, dtype=np.float64)
    return np.where(np.abs(w - w_old) >= p["dlam_min"], w, w_old), w0


def num_threads():
    return lib().or_num_threads()
