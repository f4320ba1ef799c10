"""ctypes binding of the C ABI in include/dgm.h (argument marshalling only).

Every computation happens in libdgm.so; this module converts NumPy arrays and
torch tensors to pointers and return codes to exceptions.  Importing it loads
the in-tree library and fails loudly if it has not been built.
"""

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdgm.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "libdgm.so is not built; run `python -c \"import __graft_entry__ as g; g.build()\"` "
        "or `python paper_1104_4208_gb300/build.py` first")

_lib = C.CDLL(LIB_PATH)

DGM_OK = 0
DGM_ERR = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "UNSTABLE", -5: "TIMEOUT", -6: "UNSUPPORTED"}
(DGM_ERR_INVALID_ARG, DGM_ERR_OOM, DGM_ERR_CUDA, DGM_ERR_UNSTABLE, DGM_ERR_TIMEOUT,
 DGM_ERR_UNSUPPORTED) = -1, -2, -3, -4, -5, -6
DGM_FLUX_CENTRAL, DGM_FLUX_STABILIZED = 0, 1
DGM_PREC_FP64, DGM_PREC_FP32, DGM_PREC_TC32, DGM_PREC_TC16, DGM_PREC_TCBF16, DGM_PREC_TC16X2 = 0, 1, 2, 3, 4, 5
DGM_PMAX = 8


class DgmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{DGM_ERR.get(code, code)}: {msg}")
        self.code = code


class dgm_options(C.Structure):
    _fields_ = [("flux", C.c_int), ("alpha0", C.c_double), ("precision", C.c_int),
                ("variant", C.c_int), ("checks", C.c_int), ("compensated", C.c_int),
                ("equal_order", C.c_int)]


class dgm_run_stats(C.Structure):
    _fields_ = [("h_phase_ms", C.c_double), ("e_phase_ms", C.c_double), ("other_ms", C.c_double),
                ("h_launches", C.c_int64), ("e_launches", C.c_int64), ("other_launches", C.c_int64)]


_vp = C.c_void_p
_i64 = C.c_int64
_pd = C.POINTER(C.c_double)
_pi32 = C.POINTER(C.c_int32)
_pi64 = C.POINTER(C.c_int64)

_SIGS = {
    "dgm_version": ([], C.c_int),
    "dgm_last_error": ([], C.c_char_p),
    "dgm_default_options": ([C.POINTER(dgm_options)], None),
    "dgm_create": ([C.POINTER(_vp), C.c_int], C.c_int),
    "dgm_destroy": ([_vp], C.c_int),
    "dgm_mesh_create": ([_vp, _i64, _pd, _i64, _pi32, _pi32, C.POINTER(_vp)], C.c_int),
    "dgm_mesh_destroy": ([_vp], C.c_int),
    "dgm_mesh_info": ([_vp, _pi64, _pi64, _pi64], C.c_int),
    "dgm_problem_create": ([_vp, _vp, C.c_int, _pd, _pd, C.POINTER(dgm_options), C.POINTER(_vp)], C.c_int),
    "dgm_problem_destroy": ([_vp], C.c_int),
    "dgm_problem_sizes": ([_vp, _pi64, _pi64, _pi64], C.c_int),
    "dgm_set_fields": ([_vp, _pd, _pd, _pd], C.c_int),
    "dgm_get_fields": ([_vp, _pd, _pd, _pd], C.c_int),
    "dgm_set_fields_device": ([_vp, _vp, _vp, _vp, _vp], C.c_int),
    "dgm_get_fields_device": ([_vp, _vp, _vp, _vp, _vp], C.c_int),
    "dgm_kick": ([_vp, C.c_int, C.c_double, _vp], C.c_int),
    "dgm_run": ([_vp, C.c_double, _i64, _vp, _pd], C.c_int),
    "dgm_run_composed": ([_vp, C.c_double, _i64, C.c_int, _vp], C.c_int),
    "dgm_run_timed": ([_vp, C.c_double, _i64, _vp, _pd, C.POINTER(dgm_run_stats)], C.c_int),
    "dgm_energy": ([_vp, _pd], C.c_int),
    "dgm_estimate_dt": ([_vp, C.c_int, _pd, _pd], C.c_int),
    "dgm_resonances": ([_vp, C.c_int, C.c_int, C.c_double, _pd, _pd, C.POINTER(C.c_int)], C.c_int),
    "dgm_grad_support": ([C.c_int, C.POINTER(C.c_int), _pi32, C.POINTER(C.c_int)], C.c_int),
    "dgm_grad_recurrence": ([C.c_int, C.c_int, C.POINTER(C.c_int), _pi32, _pd], C.c_int),
    "dgm_grad_sweep": ([C.c_int, C.c_int, _pd, _pd, C.POINTER(C.c_int)], C.c_int),
    "dgm_tridiag_eig": ([C.c_int, _pd, _pd, C.c_int, C.c_int, _pd, _pd], C.c_int),
    "dgm_autotune": ([_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _pd, C.POINTER(C.c_int)], C.c_int),
    "dgm_set_materials": ([_vp, _pd, _pd], C.c_int),
    "dgm_set_source": ([_vp, _pd, _pd, C.c_double, C.c_double, C.c_double], C.c_int),
    "dgm_set_time": ([_vp, C.c_double], C.c_int),
    "dgm_get_time": ([_vp, _pd], C.c_int),
    "dgm_adjoint_grad": ([_vp, C.c_double, _i64, C.c_int, _pd, C.c_int, _pd, _pd, _pd], C.c_int),
    "dgm_energy_noalloc": ([_vp, _vp, _vp], C.c_int),
    "dgm_inject_wait_timeout": ([_vp, C.c_int], C.c_int),
    "dgm_measure_fp64_peak": ([C.c_int, C.c_int, _pd], C.c_int),
    "dgm_reference_table": ([C.c_int, C.c_int, _pd, _i64, _pi64], C.c_int),
    "dgm_reference_table_2d": ([C.c_int, C.c_int, _pd, _i64, _pi64], C.c_int),
    "dgm_problem2d_create": ([_vp, _i64, _pd, _i64, _pi32, _pi32, C.c_int, _pd, _pd, C.c_int, C.POINTER(_vp)],
                             C.c_int),
    "dgm_mesh2d_info": ([_i64, _pd, _i64, _pi32, _pi32, _pi64, _pi64], C.c_int),
    "dgm_problem2d_destroy": ([_vp], C.c_int),
    "dgm_problem2d_sizes": ([_vp, _pi64, _pi64], C.c_int),
    "dgm_set_fields2d": ([_vp, _pd, _pd], C.c_int),
    "dgm_get_fields2d": ([_vp, _pd, _pd], C.c_int),
    "dgm_kick2d": ([_vp, C.c_int, C.c_double], C.c_int),
    "dgm_run2d": ([_vp, C.c_double, _i64, _vp, _pd], C.c_int),
    "dgm_quad_rule": ([C.c_int, C.POINTER(C.c_int), _pd, _pd], C.c_int),
    "dgm_batch_create": ([_vp, C.POINTER(_vp), C.c_int, C.POINTER(_vp)], C.c_int),
    "dgm_batch_destroy": ([_vp], C.c_int),
    "dgm_batch_run": ([_vp, _pd, _i64, _vp, _pd], C.c_int),
    "dgm_element_maps": ([_vp, _pd], C.c_int),
    "dgm_project_device": ([_vp, C.c_int, _vp, _vp, _vp], C.c_int),
    "dgm_eval_device": ([_vp, C.c_int, _vp, _vp, _vp], C.c_int),
    "dgm_quad_points": ([_vp, C.c_int, _pi64, _pd], C.c_int),
    "dgm_project": ([_vp, C.c_int, _pd, _pd], C.c_int),
    "dgm_eval": ([_vp, C.c_int, _pd, _pd], C.c_int),
}

for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res


def exported_symbols():
    return sorted(_SIGS)


def _check(rc):
    if rc != DGM_OK:
        raise DgmError(rc, _lib.dgm_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_pd) if a is not None else None


# ---- same names as the C ABI -------------------------------------------------
def dgm_version():
    return _lib.dgm_version()


def dgm_last_error():
    return _lib.dgm_last_error().decode()


def dgm_default_options():
    o = dgm_options()
    _lib.dgm_default_options(C.byref(o))
    return o


def dgm_create(device=0):
    h = _vp()
    _check(_lib.dgm_create(C.byref(h), device))
    return h


def dgm_destroy(ctx):
    _check(_lib.dgm_destroy(ctx))


def dgm_mesh_create(ctx, xyz, tets, vertex_key=None):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    key = None if vertex_key is None else np.ascontiguousarray(vertex_key, dtype=np.int32)
    h = _vp()
    _check(_lib.dgm_mesh_create(ctx, xyz.shape[0], _dptr(xyz), tets.shape[0],
                                tets.ctypes.data_as(_pi32),
                                None if key is None else key.ctypes.data_as(_pi32), C.byref(h)))
    return h


def dgm_mesh_destroy(mesh):
    _check(_lib.dgm_mesh_destroy(mesh))


def dgm_mesh_info(mesh):
    a, b, c = _i64(), _i64(), _i64()
    _check(_lib.dgm_mesh_info(mesh, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def dgm_problem_create(ctx, mesh, p, eps, mu, opt=None):
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    h = _vp()
    _check(_lib.dgm_problem_create(ctx, mesh, int(p), _dptr(eps), _dptr(mu),
                                   None if opt is None else C.byref(opt), C.byref(h)))
    return h


def dgm_problem_destroy(prob):
    _check(_lib.dgm_problem_destroy(prob))


def dgm_problem_sizes(prob):
    a, b, c = _i64(), _i64(), _i64()
    _check(_lib.dgm_problem_sizes(prob, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def dgm_set_fields(prob, E=None, H=None, HF=None):
    E = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
    H = None if H is None else np.ascontiguousarray(H, dtype=np.float64)
    HF = None if HF is None else np.ascontiguousarray(HF, dtype=np.float64)
    _check(_lib.dgm_set_fields(prob, _dptr(E), _dptr(H), _dptr(HF)))


def dgm_get_fields(prob, E, H, HF=None):
    _check(_lib.dgm_get_fields(prob, _dptr(E), _dptr(H), _dptr(HF)))


def dgm_set_fields_device(prob, E_ptr, H_ptr, HF_ptr=None, stream=None):
    _check(_lib.dgm_set_fields_device(prob, E_ptr, H_ptr, HF_ptr, stream))


def dgm_get_fields_device(prob, E_ptr, H_ptr, HF_ptr=None, stream=None):
    _check(_lib.dgm_get_fields_device(prob, E_ptr, H_ptr, HF_ptr, stream))


def dgm_kick(prob, which, dt, stream=None):
    _check(_lib.dgm_kick(prob, int(which), float(dt), stream))


def dgm_run(prob, dt, nsteps, stream=None, energy_out=None):
    _check(_lib.dgm_run(prob, float(dt), int(nsteps), stream, _dptr(energy_out)))


def dgm_run_timed(prob, dt, nsteps, stream=None, energy_out=None):
    st = dgm_run_stats()
    _check(_lib.dgm_run_timed(prob, float(dt), int(nsteps), stream, _dptr(energy_out), C.byref(st)))
    return st


def dgm_estimate_dt(prob, iters=50):
    rho, dt = C.c_double(), C.c_double()
    _check(_lib.dgm_estimate_dt(prob, int(iters), C.byref(rho), C.byref(dt)))
    return rho.value, dt.value


def dgm_resonances(prob, m=300, nev=8, zero_rel=1e-8):
    """-> (omega, relative residuals): up to nev smallest nonzero resonance frequencies."""
    om = np.empty(int(nev))
    res = np.empty(int(nev))
    nf = C.c_int()
    _check(_lib.dgm_resonances(prob, int(m), int(nev), float(zero_rel), _dptr(om), _dptr(res), C.byref(nf)))
    return om[:nf.value].copy(), res[:nf.value].copy()


def dgm_tridiag_eig(d, e, i0, i1, vectors=False):
    """Host-only: eigenvalues [i0, i1) of the symmetric tridiagonal (d, e), optionally unit eigenvectors."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    e = np.ascontiguousarray(e, dtype=np.float64)
    k = d.shape[0]
    vals = np.empty(int(i1) - int(i0))
    vecs = np.empty((int(i1) - int(i0), k)) if vectors else None
    _check(_lib.dgm_tridiag_eig(k, _dptr(d), _dptr(e) if k > 1 else None, int(i0), int(i1), _dptr(vals),
                                _dptr(vecs) if vectors else None))
    return (vals, vecs) if vectors else vals


AUTOTUNE_MAX = 12


def dgm_autotune(prob, steps=5):
    """-> (configs, ms_per_step, chosen index): blocks (CUDA-core) or CTAs
    (tensor-core) per SM of each candidate, its time per step, the one kept."""
    n = C.c_int()
    cfg = (C.c_int * AUTOTUNE_MAX)()
    ms = (C.c_double * AUTOTUNE_MAX)()
    ch = C.c_int()
    _check(_lib.dgm_autotune(prob, int(steps), C.byref(n), cfg, ms, C.byref(ch)))
    return list(cfg[:n.value]), list(ms[:n.value]), ch.value


def dgm_set_source(prob, xs, direction, t0, tau, amp):
    xs = np.ascontiguousarray(xs, dtype=np.float64)
    d = np.ascontiguousarray(direction, dtype=np.float64)
    _check(_lib.dgm_set_source(prob, _dptr(xs), _dptr(d), float(t0), float(tau), float(amp)))


def dgm_set_time(prob, t):
    _check(_lib.dgm_set_time(prob, float(t)))


def dgm_get_time(prob):
    t = C.c_double()
    _check(_lib.dgm_get_time(prob, C.byref(t)))
    return t.value


def dgm_set_materials(prob, eps, mu):
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    _check(_lib.dgm_set_materials(prob, _dptr(eps), _dptr(mu)))


def dgm_adjoint_grad(prob, dt, nsteps, xobs, ckpt_every, nt, mu_grad=False):
    """-> (J, dJ/d eps) or, with mu_grad, (J, dJ/d eps, dJ/d mu)."""
    xobs = np.ascontiguousarray(xobs, dtype=np.float64).reshape(-1, 3)
    J = C.c_double()
    g = np.empty(nt)
    gm = np.empty(nt) if mu_grad else None
    _check(_lib.dgm_adjoint_grad(prob, float(dt), int(nsteps), xobs.shape[0], _dptr(xobs), int(ckpt_every),
                                 C.byref(J), _dptr(g), _dptr(gm) if mu_grad else None))
    return (J.value, g, gm) if mu_grad else (J.value, g)


def dgm_energy(prob):
    w = C.c_double()
    _check(_lib.dgm_energy(prob, C.byref(w)))
    return w.value


def dgm_energy_noalloc(prob, W_device_ptr, stream=None):
    _check(_lib.dgm_energy_noalloc(prob, W_device_ptr, stream))


def dgm_inject_wait_timeout(prob, nlaunches):
    _check(_lib.dgm_inject_wait_timeout(prob, int(nlaunches)))


def dgm_measure_fp64_peak(device=0, repeats=5):
    """-> measured FP64 FMA rate of the device in TFLOP/s."""
    t = C.c_double()
    _check(_lib.dgm_measure_fp64_peak(int(device), int(repeats), C.byref(t)))
    return t.value


def dgm_reference_table(p, which):
    need = _i64()
    _check(_lib.dgm_reference_table(int(p), int(which), None, 0, C.byref(need)))
    out = np.empty(need.value)
    _check(_lib.dgm_reference_table(int(p), int(which), _dptr(out), need.value, C.byref(need)))
    return out


def dgm_reference_table_2d(p, which):
    need = _i64()
    _check(_lib.dgm_reference_table_2d(int(p), int(which), None, 0, C.byref(need)))
    out = np.empty(need.value)
    _check(_lib.dgm_reference_table_2d(int(p), int(which), _dptr(out), need.value, C.byref(need)))
    return out


def dgm_problem2d_create(ctx, xy, tris, p, eps, mu, vertex_key=None, precision=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    key = None if vertex_key is None else np.ascontiguousarray(vertex_key, dtype=np.int32)
    nt = tris.shape[0]
    eps = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (nt,)))
    mu = np.ascontiguousarray(np.broadcast_to(np.asarray(mu, dtype=np.float64), (nt,)))
    h = _vp()
    _check(_lib.dgm_problem2d_create(ctx, xy.shape[0], _dptr(xy), nt, tris.ctypes.data_as(_pi32),
                                     None if key is None else key.ctypes.data_as(_pi32), int(p), _dptr(eps),
                                     _dptr(mu), DGM_PREC_FP64 if precision is None else int(precision),
                                     C.byref(h)))
    return h


def dgm_mesh2d_info(xy, tris, vertex_key=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    key = None if vertex_key is None else np.ascontiguousarray(vertex_key, dtype=np.int32)
    a, b = _i64(), _i64()
    _check(_lib.dgm_mesh2d_info(xy.shape[0], _dptr(xy), tris.shape[0], tris.ctypes.data_as(_pi32),
                                None if key is None else key.ctypes.data_as(_pi32), C.byref(a), C.byref(b)))
    return a.value, b.value


def dgm_problem2d_destroy(prob):
    _check(_lib.dgm_problem2d_destroy(prob))


def dgm_problem2d_sizes(prob):
    a, b = _i64(), _i64()
    _check(_lib.dgm_problem2d_sizes(prob, C.byref(a), C.byref(b)))
    return a.value, b.value


def dgm_set_fields2d(prob, E=None, H=None):
    E = None if E is None else np.ascontiguousarray(E, dtype=np.float64)
    H = None if H is None else np.ascontiguousarray(H, dtype=np.float64)
    _check(_lib.dgm_set_fields2d(prob, _dptr(E), _dptr(H)))


def dgm_get_fields2d(prob, E, H):
    _check(_lib.dgm_get_fields2d(prob, _dptr(E), _dptr(H)))


def dgm_kick2d(prob, which, dt):
    _check(_lib.dgm_kick2d(prob, int(which), float(dt)))


def dgm_run2d(prob, dt, nsteps, stream=None, energies=False):
    W = np.empty(int(nsteps) + 1) if energies else None
    _check(_lib.dgm_run2d(prob, float(dt), int(nsteps), stream, _dptr(W)))
    return W


def dgm_quad_rule(q1d):
    nq = C.c_int()
    _check(_lib.dgm_quad_rule(int(q1d), C.byref(nq), None, None))
    xh = np.empty((nq.value, 3))
    w = np.empty(nq.value)
    _check(_lib.dgm_quad_rule(int(q1d), C.byref(nq), _dptr(xh), _dptr(w)))
    return xh, w


def dgm_element_maps(mesh, nt):
    out = np.empty((nt, 12))
    _check(_lib.dgm_element_maps(mesh, _dptr(out)))
    return out


def dgm_project_device(prob, q1d, E_ptr, H_ptr, stream=None):
    _check(_lib.dgm_project_device(prob, int(q1d), E_ptr, H_ptr, stream))


def dgm_eval_device(prob, q1d, E_ptr, H_ptr, stream=None):
    _check(_lib.dgm_eval_device(prob, int(q1d), E_ptr, H_ptr, stream))


def dgm_batch_create(ctx, probs):
    arr = (_vp * len(probs))(*[p.value if isinstance(p, _vp) else p for p in probs])
    h = _vp()
    _check(_lib.dgm_batch_create(ctx, arr, len(probs), C.byref(h)))
    return h


def dgm_batch_destroy(batch):
    _check(_lib.dgm_batch_destroy(batch))


def dgm_batch_run(batch, dts, nsteps, stream=None, energy_out=None):
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    _check(_lib.dgm_batch_run(batch, _dptr(dts), int(nsteps), stream, _dptr(energy_out)))


def dgm_quad_points(prob, q1d, nt):
    """-> physical quadrature points [nt][nq][3] of the rule with q1d points per direction."""
    count = _i64()
    _check(_lib.dgm_quad_points(prob, int(q1d), C.byref(count), None))
    out = np.empty(count.value)
    _check(_lib.dgm_quad_points(prob, int(q1d), C.byref(count), _dptr(out)))
    return out.reshape(nt, -1, 3)


def dgm_project(prob, q1d, E_pts, H_pts=None):
    E = np.ascontiguousarray(E_pts, dtype=np.float64) if E_pts is not None else None
    H = np.ascontiguousarray(H_pts, dtype=np.float64) if H_pts is not None else None
    _check(_lib.dgm_project(prob, int(q1d), _dptr(E), _dptr(H)))


def dgm_eval(prob, q1d, nt, want_E=True, want_H=False):
    """-> (E_pts, H_pts) [nt][nq][3] each (None where not wanted)."""
    nq = int(q1d) ** 3
    E = np.empty((nt, nq, 3)) if want_E else None
    H = np.empty((nt, nq, 3)) if want_H else None
    _check(_lib.dgm_eval(prob, int(q1d), _dptr(E), _dptr(H)))
    return E, H


def dgm_run_composed(prob, dt, nsteps, order=4, stream=None):
    _check(_lib.dgm_run_composed(prob, float(dt), int(nsteps), int(order), stream))


def dgm_grad_support(direction):
    """-> (shifts [n][4] = (di, dj, dk, carries derivative), lead position) (host only)."""
    n, lead = C.c_int(), C.c_int()
    sh = np.empty((20, 4), dtype=np.int32)
    _check(_lib.dgm_grad_support(int(direction), C.byref(n), sh.ctypes.data_as(_pi32), C.byref(lead)))
    return sh[:n.value].copy(), lead.value


def dgm_grad_recurrence(p, direction):
    """-> (ijk [n][3], coef [n][nterms]) of the derivative relations at degree p (host only)."""
    n = C.c_int()
    _check(_lib.dgm_grad_recurrence(int(p), int(direction), C.byref(n), None, None))
    nterms = len(dgm_grad_support(direction)[0])
    ijk = np.empty((n.value, 3), dtype=np.int32)
    coef = np.empty((n.value, nterms))
    _check(_lib.dgm_grad_recurrence(int(p), int(direction), C.byref(n), ijk.ctypes.data_as(_pi32), _dptr(coef)))
    return ijk, coef


def dgm_grad_sweep(p, direction, a):
    """-> (b, swept): derivative of sum a_ijk phi_ijk by the recurrence sweep (host only)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    nh = p * (p + 1) * (p + 2) // 6
    b = np.empty(nh)
    sw = C.c_int()
    _check(_lib.dgm_grad_sweep(int(p), int(direction), _dptr(a), _dptr(b), C.byref(sw)))
    return b, sw.value
