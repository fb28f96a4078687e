"""GB300 (sm_103a) adaptive-precision EAM+ACE force evaluation and MD step.

Python binding of the C ABI in include/ap.h.  Every step of the force evaluation runs
in the CUDA kernels of libapforce.so; this module only marshals arguments.  PyTorch is
used, when given, for device memory and streams (tensors are passed by pointer).

    ctx = APContext(eam, ace, box, x, v=None, fixed=None, region=None, indenter=None,
                    ind_vel=None, mass=183.84)
    f = ctx.compute_forces()          # (n, 3) float32 on the host
    ctx.step(100, 1.0)                # velocity Verlet, dt in fs
    rep = ctx.energy()                # totals of the last evaluation

Weights: w_i is the ACE weight; the paper's switching parameter is lambda_i = 1 - w_i.
"""
import ctypes as C

import numpy as np

from . import _capi
from ._capi import PRECISION, REGION, STAGES, STATUS

__all__ = ["APContext", "APError", "build", "PRECISION", "STAGES", "potential_struct", "gaunt_real",
           "eam_table_eval", "step_batch", "compute_forces_batch", "footprint_bytes", "probe_fp32_peak"]


class APError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def build(force=False, verbose=False):
    from .buildlib import build as _b
    return _b(force=force, verbose=verbose)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def potential_struct(eam, ace, mass, skin=1.0, precision="fp32", list_sizing="counted"):
    """Fill the ap_potential struct; returns (struct, keep-alive arrays).  list_sizing:
    "counted" (ap_init sizes the neighbour list by a counting pass and synchronises once) or
    "bound" (the 0.1 atoms / A^3 bound; ap_init does not wait)."""
    p = _capi.Potential()
    p.eam_n_phi = len(eam["phi_a"])
    p.eam_n_rho = len(eam["rho_a"])
    for k in range(p.eam_n_phi):
        p.eam_phi_a[k] = float(eam["phi_a"][k])
        p.eam_phi_d[k] = float(eam["phi_d"][k])
    for k in range(p.eam_n_rho):
        p.eam_rho_a[k] = float(eam["rho_a"][k])
        p.eam_rho_d[k] = float(eam["rho_d"][k])
    p.eam_rho_rclamp = float(eam.get("rho_rclamp", 0.0))
    p.eam_F_a1, p.eam_F_a2, p.eam_F_dxi = float(eam["F_a1"]), float(eam["F_a2"]), float(eam.get("F_dxi", 0.0))
    p.eam_zbl = int(eam.get("zbl", 0))
    if p.eam_zbl:
        p.eam_zbl_Z, p.eam_zbl_eps0, p.eam_zbl_a = float(eam["zbl_Z"]), float(eam["zbl_eps0"]), float(eam["zbl_a"])
        p.eam_r_lo, p.eam_r_hi = float(eam["r_lo"]), float(eam["r_hi"])
        for k in range(6):
            p.eam_b[k] = float(eam["b"][k])
    idx = np.ascontiguousarray(ace["idx"], dtype=np.int32).ravel()
    c1, c2 = _f64(ace["c1"]), _f64(ace["c2"])
    p.ace_rc, p.ace_nref = float(ace["rc"]), float(ace["nref"])
    p.ace_nmax, p.ace_lmax, p.ace_nfunc = int(ace["nmax"]), int(ace["lmax"]), len(c1)
    p.ace_idx = idx.ctypes.data_as(_capi.PI)
    p.ace_c1, p.ace_c2 = c1.ctypes.data_as(_capi.PD), c2.ctypes.data_as(_capi.PD)
    p.ace_c1_0, p.ace_c2_0 = float(ace["c1_0"]), float(ace["c2_0"])
    p.ace_precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.mass_amu = float(mass)
    p.skin = float(skin)
    p.list_sizing = {"counted": 0, "bound": 1}[list_sizing]
    return p, (idx, c1, c2)


def _box_struct(box):
    b = _capi.Box()
    h = np.asarray(box["h"], dtype=np.float64).ravel()
    for k in range(9):
        b.h[k] = h[k]
    o = box.get("origin", (0.0, 0.0, 0.0))
    for k in range(3):
        b.origin[k] = float(o[k])
        b.periodic[k] = int(box["periodic"][k])
    return b


def _region_struct(region, n):
    r = _capi.Region()
    keep = None
    if region is None:
        return r, None
    r.kind = REGION[region["kind"]]
    if region["kind"] == "sphere":
        for k in range(3):
            r.center[k] = float(region["center"][k])
        r.r_in, r.r_switch = float(region["r_in"]), float(region["r_sw"])
        r.follow_indenter = int(region.get("follow", 0))
    elif region["kind"] == "explicit":
        keep = _f64(region["w"])
        assert keep.shape == (n,)
        r.w_explicit = keep.ctypes.data_as(_capi.PD)
    elif region["kind"] == "const":
        r.w_const = float(region["w"])
    return r, keep


def _indenter_struct(ind, vel):
    s = _capi.Indenter()
    if ind is None:
        return s
    s.enabled = 1
    v = (0.0, 0.0, 0.0) if vel is None else vel
    for k in range(3):
        s.center0[k] = float(ind["center"][k])
        s.vel[k] = float(v[k])
        s.dir[k] = float(ind.get("dir", (0.0, 0.0, -1.0))[k])
    s.R, s.K = float(ind["R"]), float(ind["K"])
    return s


def _ptr(t):
    """Device pointer of a torch tensor, or None."""
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class APContext:
    """One structure on the current CUDA device (wraps ap_init / ap_destroy)."""

    def __init__(self, eam, ace, box, x, v=None, fixed=None, region=None, indenter=None, ind_vel=None,
                 mass=1.0, skin=1.0, precision="fp32", stream=None, list_sizing="counted"):
        L = _capi.lib()
        x = _f64(x, (-1, 3))
        self.n = x.shape[0]
        pot, keep = potential_struct(eam, ace, mass, skin, precision, list_sizing)
        bs = _box_struct(box)
        rs, rkeep = _region_struct(region, self.n)
        ins = _indenter_struct(indenter, ind_vel)
        vv = None if v is None else _f64(v, (-1, 3))
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8)
        h = C.c_void_p()
        st = L.ap_init(C.byref(pot), C.byref(bs), C.byref(rs), C.byref(ins), self.n,
                       x.ctypes.data_as(_capi.PD), None if vv is None else vv.ctypes.data_as(_capi.PD),
                       None if fx is None else fx.ctypes.data_as(C.POINTER(C.c_ubyte)), _stream(stream),
                       C.byref(h))
        del keep, rkeep
        if st != 0:
            raise APError(st, L.ap_last_error(None).decode())
        self._h = h
        self._L = L
        self.stream = stream          # kept alive for the context's lifetime

    def _chk(self, st):
        if st != 0:
            raise APError(st, self._L.ap_last_error(self._h).decode())

    def compute_forces(self, pos=None, out=None, stream=None):
        """Device path: pos / out are CUDA torch tensors ((n,3) float64 / float32) or None."""
        self._chk(self._L.ap_compute_forces(self._h, _ptr(pos), _ptr(out), _stream(stream)))
        return out

    def compute_forces_host(self, pos=None, out=None, stream=None):
        """Host path: numpy (n,3) float64 in, (n,3) float32 out; returns (forces, energy)."""
        if out is None:
            out = np.empty((self.n, 3), dtype=np.float32)
        e = C.c_double()
        p = None if pos is None else _f64(pos, (-1, 3))
        self._chk(self._L.ap_compute_forces_host(self._h, None if p is None else p.ctypes.data_as(_capi.PD),
                                                 out.ctypes.data_as(_capi.PF), C.byref(e), _stream(stream)))
        return out, e.value

    def step(self, n_steps, dt, stream=None):
        self._chk(self._L.ap_step(self._h, int(n_steps), float(dt), _stream(stream)))

    def energy(self, e_atom=None):
        r = _capi.Report()
        self._chk(self._L.ap_energy(self._h, C.byref(r), _ptr(e_atom)))
        return {"e_total": r.e_total, "e_pot": r.e_pot, "e_ind": r.e_ind, "e_kin": r.e_kin,
                "virial": np.array(r.virial[:]), "load": r.load, "time_fs": r.time_fs, "step": r.step,
                "n_ace": r.n_ace, "n_atoms": r.n_atoms, "e_thermostat": r.e_thermostat}

    def check(self):
        self._chk(self._L.ap_check(self._h))

    def forces(self):
        f = np.empty((self.n, 3), dtype=np.float32)
        self._chk(self._L.ap_get_forces(self._h, f.ctypes.data_as(_capi.PF)))
        return f

    def weights(self):
        w = np.empty(self.n)
        self._chk(self._L.ap_get_weights(self._h, w.ctypes.data_as(_capi.PD)))
        return w

    def set_weights(self, w):
        w = _f64(w)
        self._chk(self._L.ap_set_weights(self._h, w.ctypes.data_as(_capi.PD)))

    def get_state(self):
        x = np.empty((self.n, 3))
        v = np.empty((self.n, 3))
        t = C.c_double()
        self._chk(self._L.ap_get_state(self._h, x.ctypes.data_as(_capi.PD), v.ctypes.data_as(_capi.PD), C.byref(t)))
        return x, v, t.value

    def set_state(self, x=None, v=None, t=0.0):
        xx = None if x is None else _f64(x, (-1, 3))
        vv = None if v is None else _f64(v, (-1, 3))
        self._chk(self._L.ap_set_state(self._h, None if xx is None else xx.ctypes.data_as(_capi.PD),
                                       None if vv is None else vv.ctypes.data_as(_capi.PD), float(t)))

    def set_box(self, box):
        """Replace the box (dict with h, origin, periodic); the next evaluation re-bins."""
        b = _box_struct(box)
        self._chk(self._L.ap_set_box(self._h, C.byref(b)))

    def profile(self, enable=True):
        """Stage timing: True / 1 every stage, 2 the ACE contraction only, 3 the ACE contraction
        of one step in eight, False / 0 off."""
        self._chk(self._L.ap_profile(self._h, int(enable)))

    def profile_read(self):
        ms = (C.c_double * len(STAGES))()
        nl = (C.c_longlong * len(STAGES))()
        self._chk(self._L.ap_profile_read(self._h, ms, nl))
        return {s: (ms[k], nl[k]) for k, s in enumerate(STAGES)}

    def set_thermostat(self, t_target=None, tau_fs=100.0, group=None, kind="nose-hoover", seed=0, zero_every=0):
        """Thermostat on `group` (host mask, None = all free atoms) at t_target K with damping
        time tau_fs (ap_set_thermostat): kind "nose-hoover" or "langevin" (seed, zero_every);
        t_target None removes it."""
        t = _capi.Thermostat()
        t.kind = 0 if t_target is None else {"nose-hoover": 1, "langevin": 2}[kind]
        t.t_target = float(t_target or 0.0)
        t.tau_fs = float(tau_fs)
        t.seed = int(seed)
        t.zero_every = int(zero_every)
        g = None if group is None else np.ascontiguousarray(group, dtype=np.uint8)
        self._chk(self._L.ap_set_thermostat(self._h, C.byref(t),
                                            None if g is None else g.ctypes.data_as(C.POINTER(C.c_ubyte))))

    def csp_accumulate(self, params, out=None):
        """Add the CSP of the current positions to the block sums (ap_csp_accumulate); out: an
        optional (n,) float32 CUDA tensor receiving this evaluation's CSP (-1: surface atom)."""
        p = csp_params(params)
        self._chk(self._L.ap_csp_accumulate(self._h, C.byref(p), _ptr(out)))
        return out

    def csp_update_weights(self, params):
        """Weights from the block-averaged CSP (ap_csp_update_weights); returns the seed count."""
        p = csp_params(params)
        ns = C.c_int()
        self._chk(self._L.ap_csp_update_weights(self._h, C.byref(p), C.byref(ns)))
        return ns.value

    def record_load(self, capacity):
        """Keep the load of every later MD step in a device ring of `capacity` entries
        (ap_record_load); 0 stops."""
        self._chk(self._L.ap_record_load(self._h, int(capacity)))
        self._load_cap = int(capacity)

    def load_history(self, max_entries=None):
        """(time_fs, load) arrays of the recorded steps, oldest first (ap_load_history; one
        synchronising read-back)."""
        cap = getattr(self, "_load_cap", 0)
        if max_entries is not None:
            cap = min(cap, int(max_entries))
        t = np.empty(cap)
        p = np.empty(cap)
        cnt = C.c_int()
        self._chk(self._L.ap_load_history(self._h, t.ctypes.data_as(_capi.PD), p.ctypes.data_as(_capi.PD), cap,
                                          C.byref(cnt)))
        return t[:cnt.value].copy(), p[:cnt.value].copy()

    def memory_bytes(self):
        """Device bytes this context holds (ap_memory_bytes)."""
        return int(self._L.ap_memory_bytes(self._h))

    @property
    def launch_count(self):
        return int(self._L.ap_launch_count(self._h))

    def neighbor_info(self):
        cap = C.c_int()
        nreb = C.c_longlong()
        self._chk(self._L.ap_neighbor_info(self._h, C.byref(cap), C.byref(nreb)))
        return cap.value, nreb.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.ap_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# switching-function parameters of Appendix B (Tab. model_parameters_tungsten)
CSP_PAPER = {"csp_lo": 1.5, "csp_hi": 1.6, "r_lo": 4.0, "r_hi": 12.0, "dlam_min": 0.01, "n_avg": 110}


def csp_params(d):
    """ap_csp_params from a dict: n_nb, rc, zone_center, zone_r, and csp_lo, csp_hi, r_lo,
    r_hi, dlam_min (defaults: the paper's values)."""
    p = _capi.CspParams()
    p.n_nb = int(d["n_nb"])
    p.rc = float(d["rc"])
    p.csp_lo = float(d.get("csp_lo", CSP_PAPER["csp_lo"]))
    p.csp_hi = float(d.get("csp_hi", CSP_PAPER["csp_hi"]))
    p.r_lo = float(d.get("r_lo", CSP_PAPER["r_lo"]))
    p.r_hi = float(d.get("r_hi", CSP_PAPER["r_hi"]))
    p.dlam_min = float(d.get("dlam_min", CSP_PAPER["dlam_min"]))
    for k in range(3):
        p.zone_center[k] = float(d.get("zone_center", (0.0, 0.0, 0.0))[k])
    p.zone_r = float(d.get("zone_r", 0.0))
    return p


def step_batch(ctxs, n_steps, dt, stream=None):
    """n_steps[k] MD steps for each context ctxs[k], one kernel launch per stage for all of
    them on `stream` (ap_step_batch)."""
    L = _capi.lib()
    k = len(ctxs)
    hs = (C.c_void_p * k)(*[c._h.value for c in ctxs])
    ns = (C.c_int * k)(*[int(s) for s in n_steps])
    st = L.ap_step_batch(hs, ns, k, float(dt), _stream(stream))
    if st != 0:
        msgs = "; ".join(L.ap_last_error(c._h).decode() for c in ctxs)
        raise APError(st, msgs)


def compute_forces_batch(ctxs, stream=None):
    """One force evaluation for each context, one kernel launch per stage for all of them on
    `stream` (ap_compute_forces_batch)."""
    L = _capi.lib()
    k = len(ctxs)
    hs = (C.c_void_p * k)(*[c._h.value for c in ctxs])
    st = L.ap_compute_forces_batch(hs, k, _stream(stream))
    if st != 0:
        raise APError(st, "; ".join(L.ap_last_error(c._h).decode() for c in ctxs))


def footprint_bytes(eam, ace, n_atoms, mass=1.0, skin=1.0, ace_fraction=1.0):
    """Upper estimate of the device bytes a context of n_atoms needs (ap_footprint_bytes)."""
    pot, keep = potential_struct(eam, ace, mass, skin)
    nb = int(_capi.lib().ap_footprint_bytes(C.byref(pot), int(n_atoms), float(ace_fraction)))
    del keep
    return nb


def probe_fp32_peak(iters=200000):
    """Measured FP32 FMA throughput of the current device in TFLOP/s (ap_probe_fp32_peak)."""
    tf, ms = C.c_double(), C.c_double()
    st = _capi.lib().ap_probe_fp32_peak(int(iters), C.byref(tf), C.byref(ms))
    if st != 0:
        raise APError(st, "ap_probe_fp32_peak")
    return tf.value, ms.value


def gaunt_real(l1, m1, l2, m2, l3, m3):
    """The library's host-side real Gaunt coefficient (Racah formula route)."""
    out = C.c_double()
    st = _capi.lib().ap_gaunt_real(l1, m1, l2, m2, l3, m3, C.byref(out))
    if st != 0:
        raise APError(st, "ap_gaunt_real")
    return out.value


def eam_table_eval(eam, which, r, mass=1.0):
    """The library's EAM pair table: which 0 (Phi) / 1 (zeta) from the FP64 segments, 2 / 3 from the
    FP32 device table through the kernels' segment lookup (ap_eam_table_eval)."""
    dummy_ace = {"idx": np.zeros((0, 7), np.int32), "c1": np.zeros(0), "c2": np.zeros(0), "rc": 5.0,
                 "nref": 1.0, "nmax": 8, "lmax": 4, "c1_0": 0.0, "c2_0": 1.0}
    p, keep = potential_struct(eam, dummy_ace, mass)
    f, df = C.c_double(), C.c_double()
    st = _capi.lib().ap_eam_table_eval(C.byref(p), int(which), float(r), C.byref(f), C.byref(df))
    if st != 0:
        raise APError(st, "ap_eam_table_eval")
    return f.value, df.value
