"""ctypes binding of libpolyflood.so: argument marshalling only.

Every function named ``pf_*`` here calls the C-ABI function of the same name
(declared in include/polyflood.h); all arithmetic of the Newton step runs in
the library's CUDA kernels.  There is no CPU fallback: importing this module
when the library has not been built raises.
"""

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpolyflood.so")

PF_OK, PF_EINVAL, PF_ENOMEM, PF_ENOT_CONVERGED, PF_ETIMEOUT, PF_ECUDA, PF_EBUSY = range(7)
PF_WELL_INJECTOR, PF_WELL_PRODUCER = 0, 1
PF_DIR = {"x": 0, "y": 1, "z": 2}
PF_CTRL = {"bhp": 0, "wrate": 1, "orate": 2, "lrate": 3}
PF_PREC_FP64, PF_PREC_MIXED = 0, 1
PF_PC_BJACOBI, PF_PC_CPR = 0, 1
PF_S1_BJACOBI, PF_S1_ILU0 = 0, 1
PF_KT = {"spmv": 0, "props": 1, "face": 2, "gather": 3, "wells": 4, "ortho": 5, "precond": 6}

_STATUS = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_ENOMEM", 3: "PF_ENOT_CONVERGED", 4: "PF_ETIMEOUT",
           5: "PF_ECUDA", 6: "PF_EBUSY"}

_dp = C.POINTER(C.c_double)
_i64p = C.POINTER(C.c_int64)
_ip = C.POINTER(C.c_int)


class PfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class pf_physics(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "rho_w", "rho_o", "c_w", "c_o", "p_ref", "mu_w", "mu_o", "c_r", "p_r", "swc", "sor", "nw", "no",
        "krw_max", "kro_max", "pc_e", "pc_n", "ads_a", "ads_b", "rrf", "ipv", "omega", "mu_p0", "c_ref")] + \
        [("mixing", C.c_int), ("g", C.c_double)]


class pf_well_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_perf", C.c_int), ("cells", _i64p), ("dirs", _ip),
                ("rw", C.c_double), ("skin", C.c_double), ("gf", C.c_double), ("f", C.c_double),
                ("fh", C.c_double), ("pb0", C.c_double)]


class pf_model_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("top", C.c_double),
                ("kx", _dp), ("ky", _dp), ("kz", _dp), ("phi", _dp), ("p0", _dp), ("s0", _dp), ("c0", _dp),
                ("phys", pf_physics), ("n_wells", C.c_int), ("wells", C.POINTER(pf_well_desc)),
                ("n_sat", C.c_int), ("sat_table", _dp), ("n_poly", C.c_int), ("poly_table", _dp)]


class pf_solver_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("gmres_restart", C.c_int),
                ("gmres_max_iter", C.c_int), ("newton_max_iter", C.c_int), ("use_forcing", C.c_int),
                ("lin_rtol", C.c_double), ("newton_tol", C.c_double), ("ds_max", C.c_double),
                ("dc_frac", C.c_double),
                ("amg_pre_sweeps", C.c_int), ("amg_post_sweeps", C.c_int), ("amg_coarse_size", C.c_int),
                ("amg_cycle", C.c_int), ("autotune", C.c_int), ("forcing_form", C.c_int),
                ("stage1", C.c_int), ("amg_coarse_sweeps", C.c_int), ("reorth_eta", C.c_double),
                ("ilu_guard", C.c_double), ("newton_div", C.c_double), ("ilu_store", C.c_int),
                ("krylov_lookahead", C.c_int)]


class pf_tuning(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("props", "face", "gather", "spmv", "stage2", "rbgs", "block_cells",
                                         "ilu_fused", "cluster_cells")]


class pf_well_control(C.Structure):
    _fields_ = [("ctrl", C.c_int), ("target", C.c_double), ("limit", C.c_double), ("c_inj", C.c_double)]


class pf_iter_report(C.Structure):
    _fields_ = [("res_scaled", C.c_double), ("res_norm2", C.c_double), ("eta", C.c_double),
                ("lin_rel_res", C.c_double), ("krylov_iters", C.c_int), ("converged", C.c_int)]


class pf_step_report(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("krylov_iters", C.c_int), ("converged", C.c_int),
                ("res_scaled", C.c_double)]


class pf_period(C.Structure):
    _fields_ = [("n_steps", C.c_int), ("dt", C.c_double), ("controls", C.POINTER(pf_well_control))]


class pf_schedule(C.Structure):
    _fields_ = [("n_periods", C.c_int), ("periods", C.POINTER(pf_period))]


class pf_run_report(C.Structure):
    _fields_ = [("steps", C.c_int), ("newton_iters", C.c_int), ("krylov_iters", C.c_int), ("cuts", C.c_int),
                ("status", C.c_int), ("seconds", C.c_double)]


class pf_result(C.Structure):
    _fields_ = [("state", C.c_int), ("status", C.c_int), ("report", pf_run_report), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_end", C.c_double), ("footprint", C.c_size_t)]


PF_REQ_QUEUED, PF_REQ_RUNNING, PF_REQ_DONE, PF_REQ_FAILED = range(4)

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpolyflood.so is not built (run __graft_entry__.build() or "
                               "python -m paper_1807_05298_gb300.build); there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp = C.c_void_p
        sig = {
            "pf_version": ([], C.c_char_p),
            "pf_last_error": ([], C.c_char_p),
            "pf_default_opts": ([C.POINTER(pf_solver_opts)], C.c_int),
            "pf_create": ([C.POINTER(pf_model_desc), C.POINTER(pf_solver_opts), vp, C.POINTER(vp)], C.c_int),
            "pf_destroy": ([vp], C.c_int),
            "pf_set_controls": ([vp, C.POINTER(pf_well_control), C.c_int], C.c_int),
            "pf_begin_step": ([vp, C.c_double], C.c_int),
            "pf_newton_iteration": ([vp, C.POINTER(pf_iter_report)], C.c_int),
            "pf_step": ([vp, C.c_double, C.POINTER(pf_step_report)], C.c_int),
            "pf_assemble": ([vp], C.c_int),
            "pf_export_system": ([vp, _dp, _dp, _dp, _dp, _dp], C.c_int),
            "pf_apply_jacobian": ([vp, _dp, _dp], C.c_int),
            "pf_solve_linear": ([vp, _dp, _dp, C.c_double, _ip, _dp], C.c_int),
            "pf_get_state": ([vp, _dp, _dp, _dp, _dp], C.c_int),
            "pf_set_state": ([vp, _dp, _dp, _dp, _dp], C.c_int),
            "pf_sizes": ([vp, _i64p, _ip, _i64p], C.c_int),
            "pf_device_state": ([vp, C.POINTER(_dp)], C.c_int),
            "pf_launch_count": ([vp, _i64p], C.c_int),
            "pf_well_rates": ([vp, _dp, _dp, _dp, _dp], C.c_int),
            "pf_well_switched": ([vp, _ip], C.c_int),
            "pf_end_step": ([vp, _ip], C.c_int),
            "pf_abort_step": ([vp], C.c_int),
            "pf_get_x": ([vp, _dp], C.c_int),
            "pf_set_x": ([vp, _dp], C.c_int),
            "pf_kernel_timing_enable": ([vp, C.c_int], C.c_int),
            "pf_kernel_timing": ([vp, C.c_int, _i64p, _dp], C.c_int),
            "pf_autotune": ([vp, C.POINTER(pf_tuning)], C.c_int),
            "pf_set_tuning": ([vp, C.POINTER(pf_tuning)], C.c_int),
            "pf_get_tuning": ([vp, C.POINTER(pf_tuning)], C.c_int),
            "pf_set_programmatic_launch": ([C.c_int], C.c_int),
            "pf_inject_create_failure": ([C.c_int], C.c_int),
            "pf_apply_preconditioner": ([vp, _dp, _dp], C.c_int),
            "pf_equilibrium_init": ([C.POINTER(pf_model_desc), C.c_double, C.c_double, C.c_double, _dp, _dp],
                                    C.c_int),
            "pf_run_schedule": ([vp, C.POINTER(pf_schedule), C.c_int, C.POINTER(pf_run_report)], C.c_int),
            "pf_runtime_last_error": ([], C.c_char_p),
            "pf_footprint": ([C.POINTER(pf_model_desc), C.POINTER(pf_solver_opts), C.POINTER(C.c_size_t)],
                             C.c_int),
            "pf_batch_create": ([C.POINTER(C.POINTER(pf_model_desc)), C.c_int, C.POINTER(pf_solver_opts), C.c_int,
                                 C.POINTER(vp)], C.c_int),
            "pf_batch_run": ([vp, C.POINTER(C.POINTER(pf_schedule)), C.c_int, C.POINTER(pf_run_report)], C.c_int),
            "pf_batch_member": ([vp, C.c_int, C.POINTER(vp)], C.c_int),
            "pf_batch_destroy": ([vp], C.c_int),
            "pf_batch_set_packing": ([vp, C.c_int, C.c_double], C.c_int),
            "pf_batch_packing_stats": ([vp, _i64p, _i64p], C.c_int),
            "pf_server_create": ([C.c_size_t, C.c_int, C.POINTER(pf_solver_opts), C.c_int, C.POINTER(vp)],
                                 C.c_int),
            "pf_server_submit": ([vp, C.POINTER(pf_model_desc), C.POINTER(pf_schedule), C.POINTER(C.c_uint64)],
                                 C.c_int),
            "pf_server_poll": ([vp, C.c_uint64, C.POINTER(pf_result)], C.c_int),
            "pf_server_wait": ([vp, C.c_uint64, C.c_double, C.POINTER(pf_result)], C.c_int),
            "pf_server_fetch_state": ([vp, C.c_uint64, _dp, _dp, _dp, _dp], C.c_int),
            "pf_server_stats": ([vp, C.POINTER(C.c_size_t), _ip, _ip], C.c_int),
            "pf_server_destroy": ([vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in dir(lib()) if n.startswith("pf_")]


def _check(rc):
    if rc != PF_OK:
        raise PfError(rc, lib().pf_last_error().decode())
    return rc


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def default_opts(**over):
    o = pf_solver_opts()
    _check(lib().pf_default_opts(C.byref(o)))
    for k, v in over.items():
        setattr(o, k, v)
    return o


def physics_struct(ph):
    p = pf_physics()
    for name, _ in pf_physics._fields_:
        setattr(p, name, int(ph[name]) if name == "mixing" else float(ph[name]))
    return p


class Model:
    """pf_model_desc built from a scenario dict (keeps the arrays alive)."""

    def __init__(self, sc):
        self.keep = []
        arr = lambda a: self._keep(np.ascontiguousarray(a, dtype=np.float64))
        d = pf_model_desc()
        d.nx, d.ny, d.nz = sc["nx"], sc["ny"], sc["nz"]
        d.dx, d.dy, d.dz, d.top = sc["dx"], sc["dy"], sc["dz"], sc["top"]
        d.kx, d.ky, d.kz = _ptr(arr(sc["kx"])), _ptr(arr(sc["ky"])), _ptr(arr(sc["kz"]))
        d.phi = _ptr(arr(sc["phi"]))
        d.p0, d.s0, d.c0 = _ptr(arr(sc["P0"])), _ptr(arr(sc["S0"])), _ptr(arr(sc["C0"]))
        d.phys = physics_struct(sc["physics"])
        nw = len(sc["wells"])
        wells = (pf_well_desc * max(1, nw))()
        for i, w in enumerate(sc["wells"]):
            cells = self._keep(np.ascontiguousarray(w["cells"], dtype=np.int64))
            dirs = self._keep(np.ascontiguousarray([PF_DIR[x] for x in w["dirs"]], dtype=np.int32))
            wd = wells[i]
            wd.kind = PF_WELL_INJECTOR if w["kind"] == "inj" else PF_WELL_PRODUCER
            wd.n_perf = len(cells)
            wd.cells = cells.ctypes.data_as(_i64p)
            wd.dirs = dirs.ctypes.data_as(_ip)
            wd.rw, wd.skin, wd.gf, wd.f, wd.fh = w["rw"], w["skin"], w["gf"], w["f"], w["fh"]
            wd.pb0 = w["Pb0"]
        self.keep.append(wells)
        d.n_wells = nw
        d.wells = C.cast(wells, C.POINTER(pf_well_desc))
        ph = sc["physics"]
        if ph.get("sat_table") is not None:
            t = arr(np.asarray(ph["sat_table"], dtype=np.float64).reshape(-1, 4))
            d.n_sat, d.sat_table = t.shape[0], _ptr(t)
        if ph.get("poly_table") is not None:
            t = arr(np.asarray(ph["poly_table"], dtype=np.float64).reshape(-1, 3))
            d.n_poly, d.poly_table = t.shape[0], _ptr(t)
        self.desc = d

    def _keep(self, a):
        self.keep.append(a)
        return a


def inject_create_failure(k):
    """Arms the host-side fault injection of the next pf_create: its k-th CUDA
    call reports an error instead of running (k = 0 disarms)."""
    _check(lib().pf_inject_create_failure(int(k)))


def set_programmatic_launch(on):
    """Process-wide switch for programmatic dependent launch (default off)."""
    _check(lib().pf_set_programmatic_launch(1 if on else 0))


def equilibrium_init(sc, datum_depth, datum_p, contact_depth):
    """Capillary-gravity equilibrium (P_o, S_w) per cell for the scenario's
    grid, rock and fluids (pf_equilibrium_init; host code in the library)."""
    m = Model(dict(sc, P0=np.zeros(sc["nx"] * sc["ny"] * sc["nz"]), S0=np.zeros(sc["nx"] * sc["ny"] * sc["nz"]),
                   C0=np.zeros(sc["nx"] * sc["ny"] * sc["nz"])))
    n = sc["nx"] * sc["ny"] * sc["nz"]
    P = np.empty(n)
    S = np.empty(n)
    _check(lib().pf_equilibrium_init(C.byref(m.desc), float(datum_depth), float(datum_p), float(contact_depth),
                                     _ptr(P), _ptr(S)))
    return P, S


def controls_array(controls):
    arr = (pf_well_control * max(1, len(controls)))()
    for i, c in enumerate(controls):
        arr[i].ctrl = PF_CTRL[c["ctrl"]]
        arr[i].target = c["target"]
        arr[i].limit = 0.0 if c.get("limit") is None else c["limit"]
        arr[i].c_inj = c.get("c_inj", 0.0)
    return arr


def current_stream_handle():
    """cudaStream_t of torch's current stream (torch provides streams only)."""
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Simulator:
    """One pf_sim: a scenario resident on the current CUDA device."""

    def __init__(self, sc, opts=None, stream=None, **opt_over):
        self.sc = sc
        self.model = Model(sc)
        self.opts = opts if opts is not None else default_opts(**opt_over)
        h = C.c_void_p()
        _check(lib().pf_create(C.byref(self.model.desc), C.byref(self.opts), stream, C.byref(h)))
        self.h = h
        n = C.c_int64(); nw = C.c_int(); npf = C.c_int64()
        _check(lib().pf_sizes(h, C.byref(n), C.byref(nw), C.byref(npf)))
        self.n, self.nw, self.npf = n.value, nw.value, npf.value
        self.nunk = 3 * self.n + self.nw

    def close(self):
        if self.h:
            lib().pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_controls(self, controls):
        arr = controls_array(controls)
        _check(lib().pf_set_controls(self.h, arr, len(controls)))

    def begin_step(self, dt):
        _check(lib().pf_begin_step(self.h, dt))

    def newton_iteration(self):
        r = pf_iter_report()
        _check(lib().pf_newton_iteration(self.h, C.byref(r)))
        return r

    def step(self, dt, raise_on_failure=True):
        r = pf_step_report()
        rc = lib().pf_step(self.h, dt, C.byref(r))
        if rc != PF_OK and (raise_on_failure or rc != PF_ENOT_CONVERGED):
            _check(rc)
        return rc, r

    def assemble(self):
        _check(lib().pf_assemble(self.h))

    def export_system(self):
        R = np.empty(self.nunk)
        Jc = np.empty(7 * 9 * self.n)
        Bw = np.empty(max(1, 3 * self.npf))
        Cw = np.empty(max(1, 3 * self.npf))
        Dw = np.empty(max(1, self.nw))
        _check(lib().pf_export_system(self.h, _ptr(R), _ptr(Jc), _ptr(Bw), _ptr(Cw), _ptr(Dw)))
        return R, Jc.reshape(7, 9, self.n), Bw[:3 * self.npf].reshape(3, self.npf), \
            Cw[:3 * self.npf].reshape(3, self.npf), Dw[:self.nw]

    def export_residual(self):
        """R alone (pf_export_system with the Jacobian outputs skipped)."""
        R = np.empty(self.nunk)
        _check(lib().pf_export_system(self.h, _ptr(R), None, None, None, None))
        return R

    def apply_jacobian(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.nunk)
        _check(lib().pf_apply_jacobian(self.h, _ptr(x), _ptr(y)))
        return y

    def apply_preconditioner(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        z = np.empty(self.nunk)
        _check(lib().pf_apply_preconditioner(self.h, _ptr(v), _ptr(z)))
        return z

    def solve_linear(self, b, rtol):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty(self.nunk)
        its = C.c_int()
        rr = C.c_double()
        _check(lib().pf_solve_linear(self.h, _ptr(b), _ptr(x), rtol, C.byref(its), C.byref(rr)))
        return x, its.value, rr.value

    def get_state(self):
        P, S, Cc, Pb = (np.empty(self.n), np.empty(self.n), np.empty(self.n), np.empty(max(1, self.nw)))
        _check(lib().pf_get_state(self.h, _ptr(P), _ptr(S), _ptr(Cc), _ptr(Pb)))
        return P, S, Cc, Pb[:self.nw]

    def get_x(self, out=None):
        """State as the block-wise unknown vector [P,S,C per cell..., Pb per well]."""
        x = np.empty(self.nunk) if out is None else out
        _check(lib().pf_get_x(self.h, _ptr(x)))
        return x

    def get_x_ptr(self, addr):
        """pf_get_x into caller memory at address ``addr`` (e.g. a pinned tensor)."""
        _check(lib().pf_get_x(self.h, C.cast(C.c_void_p(addr), _dp)))

    def set_x_ptr(self, addr):
        _check(lib().pf_set_x(self.h, C.cast(C.c_void_p(addr), _dp)))

    def end_step(self):
        r = C.c_int()
        _check(lib().pf_end_step(self.h, C.byref(r)))
        return bool(r.value)

    def abort_step(self):
        _check(lib().pf_abort_step(self.h))

    def autotune(self):
        t = pf_tuning()
        _check(lib().pf_autotune(self.h, C.byref(t)))
        return {n: getattr(t, n) for n, _ in pf_tuning._fields_}

    def tuning(self):
        t = pf_tuning()
        _check(lib().pf_get_tuning(self.h, C.byref(t)))
        return {n: getattr(t, n) for n, _ in pf_tuning._fields_}

    def set_tuning(self, **shapes):
        t = pf_tuning()
        cur = dict(props=256, face=256, gather=256, spmv=256, stage2=256, rbgs=256,
                   block_cells=4096 if self.opts.precision == PF_PREC_MIXED else 512, ilu_fused=1,
                   cluster_cells=0)
        cur.update(shapes)
        for k, v in cur.items():
            setattr(t, k, int(v))
        _check(lib().pf_set_tuning(self.h, C.byref(t)))

    def kernel_timing_enable(self, on=True):
        _check(lib().pf_kernel_timing_enable(self.h, 1 if on else 0))

    def kernel_timing(self, which):
        c = C.c_int64(); ms = C.c_double()
        _check(lib().pf_kernel_timing(self.h, PF_KT[which], C.byref(c), C.byref(ms)))
        return c.value, ms.value

    def set_state(self, P=None, S=None, Cc=None, Pb=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        P, S, Cc, Pb = f(P), f(S), f(Cc), f(Pb)
        _check(lib().pf_set_state(self.h, _ptr(P), _ptr(S), _ptr(Cc), _ptr(Pb)))

    def set_x(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        _check(lib().pf_set_x(self.h, _ptr(x)))

    def well_rates(self):
        """(q_w, q_o, q_p, Pb) per well: mass rates into the reservoir [kg/s]."""
        q = [np.empty(max(1, self.nw)) for _ in range(4)]
        _check(lib().pf_well_rates(self.h, *[_ptr(a) for a in q]))
        return tuple(a[:self.nw] for a in q)

    def switched(self):
        out = np.zeros(max(1, self.nw), dtype=np.int32)
        _check(lib().pf_well_switched(self.h, out.ctypes.data_as(_ip)))
        return out[:self.nw].astype(bool)

    def launch_count(self):
        c = C.c_int64()
        _check(lib().pf_launch_count(self.h, C.byref(c)))
        return c.value

    def run_schedule(self, n_steps=None, max_cuts=6, callback=None):
        """Fixed-step time loop over the scenario schedule; halves the step on a
        Newton failure (the library restores x^n)."""
        done = 0
        hist = []
        for period in self.sc["schedule"]:
            self.set_controls(period["controls"])
            for _ in range(period["n_steps"]):
                if n_steps is not None and done >= n_steps:
                    return hist
                left = period["dt"]
                dt = left
                cuts = 0
                newton = krylov = 0
                while left > 0.0:
                    dt = min(dt, left)
                    rc, rep = self.step(dt, raise_on_failure=False)
                    newton += rep.newton_iters
                    krylov += rep.krylov_iters
                    if rc == PF_OK:
                        left -= dt
                        dt = min(2.0 * dt, period["dt"])   # grow back after a cut
                    else:
                        cuts += 1
                        if cuts > max_cuts:
                            raise PfError(rc, "time step cut limit reached")
                        dt *= 0.5
                done += 1
                rec = dict(newton=newton, krylov=krylov, cuts=cuts)
                hist.append(rec)
                if callback is not None:
                    callback(self, rec)
        return hist


def _rt_check(rc):
    if rc != PF_OK:
        raise PfError(rc, lib().pf_runtime_last_error().decode())
    return rc


class Schedule:
    """pf_schedule built from a scenario's schedule list (keeps arrays alive);
    ``n_steps`` truncates it."""

    def __init__(self, schedule, n_steps=None):
        periods = []
        left = n_steps
        for p in schedule:
            k = p["n_steps"] if left is None else min(p["n_steps"], left)
            if k <= 0:
                break
            periods.append((k, p["dt"], controls_array(p["controls"])))
            if left is not None:
                left -= k
        self.arr = (pf_period * max(1, len(periods)))()
        self.keep = []
        for i, (k, dt, ctl) in enumerate(periods):
            self.arr[i].n_steps = k
            self.arr[i].dt = dt
            self.arr[i].controls = C.cast(ctl, C.POINTER(pf_well_control))
            self.keep.append(ctl)
        self.s = pf_schedule(len(periods), C.cast(self.arr, C.POINTER(pf_period)))
        self.n_steps = sum(p[0] for p in periods)


def run_schedule(sim, schedule, max_cuts=6):
    """Native time loop (pf_run_schedule) over a scenario schedule."""
    rep = pf_run_report()
    _rt_check(lib().pf_run_schedule(sim.h, C.byref(schedule.s), max_cuts, C.byref(rep)))
    return rep


def footprint(sc, opts=None, **over):
    m = Model(sc)
    o = opts if opts is not None else default_opts(**over)
    b = C.c_size_t()
    _check(lib().pf_footprint(C.byref(m.desc), C.byref(o), C.byref(b)))
    return b.value


class Batch:
    """Many scenarios resident at once, each with its own stream; pf_batch_run
    drives them from ``n_threads`` host threads."""

    def __init__(self, scenarios, n_threads=8, opts=None, packed=False, pack_window_us=0.0, **over):
        self.models = [Model(sc) for sc in scenarios]
        self.opts = opts if opts is not None else default_opts(**over)
        arr = (C.POINTER(pf_model_desc) * len(self.models))(*[C.pointer(m.desc) for m in self.models])
        h = C.c_void_p()
        _rt_check(lib().pf_batch_create(arr, len(self.models), C.byref(self.opts), n_threads, C.byref(h)))
        self.h = h
        self.scenarios = scenarios
        if packed:
            self.set_packing(True, pack_window_us)

    def set_packing(self, on, window_us=0.0):
        """Packed assembly (pf_batch_set_packing): one launch per assembly
        kernel over the members that reach an assembly together."""
        _rt_check(lib().pf_batch_set_packing(self.h, 1 if on else 0, float(window_us)))

    def packing_stats(self):
        """(packs launched, members assembled through them)."""
        p = C.c_int64(); m = C.c_int64()
        _rt_check(lib().pf_batch_packing_stats(self.h, C.byref(p), C.byref(m)))
        return p.value, m.value

    def run(self, n_steps=None, max_cuts=6, raise_on_failure=True):
        scheds = [Schedule(sc["schedule"], n_steps) for sc in self.scenarios]
        arr = (C.POINTER(pf_schedule) * len(scheds))(*[C.pointer(s.s) for s in scheds])
        reps = (pf_run_report * len(scheds))()
        rc = lib().pf_batch_run(self.h, arr, max_cuts, reps)
        if rc != PF_OK and raise_on_failure:
            _rt_check(rc)
        return list(reps)

    def member_x(self, i):
        p = C.c_void_p()
        _rt_check(lib().pf_batch_member(self.h, i, C.byref(p)))
        n = C.c_int64(); nw = C.c_int(); npf = C.c_int64()
        _check(lib().pf_sizes(p, C.byref(n), C.byref(nw), C.byref(npf)))
        x = np.empty(3 * n.value + nw.value)
        _check(lib().pf_get_x(p, _ptr(x)))
        return x

    def close(self):
        if self.h:
            lib().pf_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server with admission by device footprint."""

    def __init__(self, hbm_budget, n_workers=8, opts=None, max_cuts=6, **over):
        self.opts = opts if opts is not None else default_opts(**over)
        h = C.c_void_p()
        _rt_check(lib().pf_server_create(int(hbm_budget), n_workers, C.byref(self.opts), max_cuts, C.byref(h)))
        self.h = h
        self.meta = {}

    def submit(self, sc, n_steps=None):
        m = Model(sc)
        s = Schedule(sc["schedule"], n_steps)
        t = C.c_uint64()
        _rt_check(lib().pf_server_submit(self.h, C.byref(m.desc), C.byref(s.s), C.byref(t)))
        self.meta[t.value] = (sc["nx"] * sc["ny"] * sc["nz"], len(sc["wells"]))
        return t.value

    def poll(self, ticket):
        r = pf_result()
        _rt_check(lib().pf_server_poll(self.h, ticket, C.byref(r)))
        return r

    def wait(self, ticket, timeout=3600.0):
        r = pf_result()
        _rt_check(lib().pf_server_wait(self.h, ticket, timeout, C.byref(r)))
        return r

    def state(self, ticket):
        n, nw = self.meta[ticket]
        P, S, Cc, Pb = np.empty(n), np.empty(n), np.empty(n), np.empty(max(1, nw))
        _rt_check(lib().pf_server_fetch_state(self.h, ticket, _ptr(P), _ptr(S), _ptr(Cc), _ptr(Pb)))
        return P, S, Cc, Pb[:nw]

    def stats(self):
        u = C.c_size_t(); r = C.c_int(); q = C.c_int()
        _rt_check(lib().pf_server_stats(self.h, C.byref(u), C.byref(r), C.byref(q)))
        return u.value, r.value, q.value

    def close(self):
        if self.h:
            lib().pf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
