"""Indentation observables from a running context (Sec. 2.1 and 3: Eqs. P_ind, hertz_fit,
p_m, contact_radius).

The load P_ind (Eq. P_ind) of every MD step is kept on the device (ap_record_load: the
blend kernel adds each step's load to a ring buffer) and read back once per recording;
this module records it against the indentation depth and evaluates the paper's closed
forms on the series:

    depth            h = z_surf + R - z_tip(t)        (z_tip moves with the indenter velocity)
    Hertz load       P_H = 4/3 E* R^(1/2) h^(3/2)     (E* by linear least squares through 0)
    contact radius   a_c = sqrt(h (2 R - h))
    hardness         p_m = P_ind / (pi a_c^2)

Units: eV, A, fs; moduli and pressures are returned in GPa.
"""
import numpy as np

EV_PER_A3_IN_GPA = 160.21766208

__all__ = ["record_indentation", "hertz_modulus", "contact_radius", "hardness", "EV_PER_A3_IN_GPA"]


def record_indentation(ctx, indenter, ind_vel, z_surf, n_steps, every, dt=1.0, stream=None):
    """Advance ctx by n_steps MD steps and return the load of the starting state and of every
    `every`-th step (and of the last one).  The steps' loads stay on the device until one
    read-back at the end; the starting state's load comes from one ap_energy call.
    indenter: the dict the context was created with (center, R); ind_vel: its velocity (A/fs,
    moves along -z for (0, 0, v)).  Returns dict(time_fs, depth, load)."""
    R = float(indenter["R"])
    z0 = float(indenter["center"][2])
    vz = float(np.asarray(ind_vel)[2])
    rep = ctx.energy()
    ctx.record_load(max(1, n_steps))
    try:
        ctx.step(n_steps, dt, stream)
        t_all, p_all = ctx.load_history()
    finally:
        ctx.record_load(0)
    pick = list(range(every - 1, n_steps, every))
    if n_steps > 0 and (not pick or pick[-1] != n_steps - 1):
        pick.append(n_steps - 1)
    times = np.concatenate([[rep["time_fs"]], t_all[pick]])
    load = np.concatenate([[rep["load"]], p_all[pick]])
    depth = z_surf + R - (z0 - vz * times)
    return {"time_fs": times, "depth": depth, "load": load}


def hertz_modulus(depth, load, R, h_max=None):
    """E* (GPa) of Eq. hertz_fit by least squares over the points with 0 < h <= h_max."""
    h = np.asarray(depth, dtype=np.float64)
    P = np.asarray(load, dtype=np.float64)
    sel = h > 0.0
    if h_max is not None:
        sel &= h <= h_max
    x = 4.0 / 3.0 * np.sqrt(R) * h[sel] ** 1.5
    if not np.any(x > 0.0):
        raise ValueError("no positive depths to fit")
    return float((x @ P[sel]) / (x @ x)) * EV_PER_A3_IN_GPA


def contact_radius(depth, R):
    """a_c = sqrt(h (2R - h)) (Eq. contact_radius), A."""
    h = np.asarray(depth, dtype=np.float64)
    return np.sqrt(np.clip(h * (2.0 * R - h), 0.0, None))


def hardness(depth, load, R):
    """Mean contact pressure p_m = P_ind / (pi a_c^2) (Eq. p_m), GPa; NaN where a_c = 0."""
    a = contact_radius(depth, R)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(a > 0.0, np.asarray(load, dtype=np.float64) / (np.pi * a * a), np.nan) * EV_PER_A3_IN_GPA
