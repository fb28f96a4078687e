"""ctypes declarations of the C ABI in include/ap.h (argument marshalling only)."""
import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libapforce.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ap.h")

D, I, LL, SZ = C.c_double, C.c_int, C.c_longlong, C.c_size_t
PD, PF, PI, PLL = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int), C.POINTER(C.c_longlong)
VP = C.c_void_p

AP_OK, AP_ERR_ARG, AP_ERR_OOM, AP_ERR_CUDA, AP_ERR_DOMAIN, AP_ERR_CAPACITY, AP_ERR_TIMEOUT, AP_ERR_STATE = 0, -1, -2, -3, -4, -5, -6, -7
AP_ERR_LIMIT = -8
STATUS = {0: "AP_OK", -1: "AP_ERR_ARG", -2: "AP_ERR_OOM", -3: "AP_ERR_CUDA", -4: "AP_ERR_DOMAIN",
          -5: "AP_ERR_CAPACITY", -6: "AP_ERR_TIMEOUT", -7: "AP_ERR_STATE", -8: "AP_ERR_LIMIT"}
PRECISION = {"fp32": 0, "tf32x3": 1, "bf16": 2, "fp16": 3, "fp64": 4}
REGION = {None: 0, "none": 0, "sphere": 1, "explicit": 2, "const": 3}
STAGES = ["neighbor", "prepare", "eam_density", "eam_force", "ace", "blend", "integrate", "ace_basis", "ace_force"]


class Potential(C.Structure):
    _fields_ = [("eam_n_phi", I), ("eam_phi_a", D * 32), ("eam_phi_d", D * 32),
                ("eam_n_rho", I), ("eam_rho_a", D * 16), ("eam_rho_d", D * 16),
                ("eam_rho_rclamp", D), ("eam_F_a1", D), ("eam_F_a2", D), ("eam_F_dxi", D),
                ("eam_zbl", I), ("eam_zbl_Z", D), ("eam_zbl_eps0", D), ("eam_zbl_a", D),
                ("eam_r_lo", D), ("eam_r_hi", D), ("eam_b", D * 6),
                ("ace_rc", D), ("ace_nref", D), ("ace_nmax", I), ("ace_lmax", I), ("ace_nfunc", I),
                ("ace_idx", PI), ("ace_c1", PD), ("ace_c2", PD), ("ace_c1_0", D), ("ace_c2_0", D),
                ("ace_precision", I), ("mass_amu", D), ("skin", D), ("list_sizing", I)]


class Box(C.Structure):
    _fields_ = [("h", D * 9), ("origin", D * 3), ("periodic", I * 3)]


class Region(C.Structure):
    _fields_ = [("kind", I), ("center", D * 3), ("r_in", D), ("r_switch", D),
                ("follow_indenter", I), ("w_explicit", PD), ("w_const", D)]


class Indenter(C.Structure):
    _fields_ = [("enabled", I), ("center0", D * 3), ("vel", D * 3), ("R", D), ("K", D), ("dir", D * 3)]


class Report(C.Structure):
    _fields_ = [("e_total", D), ("e_pot", D), ("e_ind", D), ("e_kin", D), ("virial", D * 6),
                ("load", D), ("time_fs", D), ("step", LL), ("n_ace", I), ("n_atoms", I), ("e_thermostat", D)]


_lib = None


class Thermostat(C.Structure):
    _fields_ = [("kind", C.c_int), ("t_target", C.c_double), ("tau_fs", C.c_double), ("seed", C.c_ulonglong),
                ("zero_every", C.c_int)]


class CspParams(C.Structure):
    _fields_ = [("n_nb", C.c_int), ("rc", C.c_double), ("csp_lo", C.c_double), ("csp_hi", C.c_double),
                ("r_lo", C.c_double), ("r_hi", C.c_double), ("dlam_min", C.c_double),
                ("zone_center", C.c_double * 3), ("zone_r", C.c_double)]


def lib():
    """Load libapforce.so; raise if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise RuntimeError("libapforce.so is not built: run `python -m paper_2505_12958_gb300.buildlib` "
                           "(nvcc for sm_103a) first")
    L = C.CDLL(LIBPATH)
    P = C.POINTER
    sig = {
        "ap_init": (I, [P(Potential), P(Box), P(Region), P(Indenter), I, PD, PD, C.POINTER(C.c_ubyte), VP, P(VP)]),
        "ap_compute_forces": (I, [VP, VP, VP, VP]),
        "ap_compute_forces_host": (I, [VP, PD, PF, PD, VP]),
        "ap_step": (I, [VP, I, D, VP]),
        "ap_step_batch": (I, [C.POINTER(VP), PI, I, D, VP]),
        "ap_compute_forces_batch": (I, [C.POINTER(VP), I, VP]),
        "ap_csp_accumulate": (I, [VP, P(CspParams), VP]),
        "ap_set_thermostat": (I, [VP, P(Thermostat), C.POINTER(C.c_ubyte)]),
        "ap_csp_update_weights": (I, [VP, P(CspParams), PI]),
        "ap_memory_bytes": (C.c_size_t, [VP]),
        "ap_energy": (I, [VP, P(Report), VP]),
        "ap_check": (I, [VP]),
        "ap_get_state": (I, [VP, PD, PD, PD]),
        "ap_set_state": (I, [VP, PD, PD, D]),
        "ap_get_forces": (I, [VP, PF]),
        "ap_set_box": (I, [VP, P(Box)]),
        "ap_get_weights": (I, [VP, PD]),
        "ap_set_weights": (I, [VP, PD]),
        "ap_profile": (I, [VP, I]),
        "ap_profile_read": (I, [VP, PD, PLL]),
        "ap_launch_count": (LL, [VP]),
        "ap_neighbor_info": (I, [VP, PI, PLL]),
        "ap_footprint_bytes": (SZ, [P(Potential), I, D]),
        "ap_last_error": (C.c_char_p, [VP]),
        "ap_inject_alloc_failures": (None, [I]),
        "ap_record_load": (I, [VP, I]),
        "ap_load_history": (I, [VP, PD, PD, I, PI]),
        "ap_destroy": (None, [VP]),
        "ap_version": (I, []),
        "ap_ace_forces_noalloc": (I, [P(Potential), I, I, VP, VP, VP, VP, VP, VP]),
        "ap_gaunt_real": (I, [I, I, I, I, I, I, PD]),
        "ap_probe_fp32_peak": (I, [I, PD, PD]),
        "ap_eam_table_eval": (I, [P(Potential), I, D, PD, PD]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def header_symbols():
    """Names of the functions include/ap.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ap_[a-z_0-9]+)\s*\(", txt)))
