"""ctypes binding of libpff (argument marshalling only; every computation runs in the CUDA library).

Vectors are torch tensors on the CUDA device, contiguous, float64 (or float32 where a precision
argument says 32), in the component-blocked DoF layout [u_1 | ... | u_d | phi] of include/pff.h.
"""
import ctypes
import os

import torch

from . import build as _build

PFF_SPLIT_NONE, PFF_SPLIT_MIEHE = 0, 1
PFF_MODE_FULL, PFF_MODE_BLOCKDIAG, PFF_MODE_TRANSPOSE = 0, 1, 2
PFF_MASK_RAW, PFF_MASK_ADJOINT = 4, 8
PFF_FLAG_TOP, PFF_FLAG_BOTTOM, PFF_FLAG_SLIT, PFF_FLAG_COPY = 0x10, 0x20, 0x40, 0x80
PFF_PROF_OFF, PFF_PROF_JAC64_L0, PFF_PROF_JAC32_L0, PFF_PROF_JAC64, PFF_PROF_JAC32, PFF_PROF_RESIDUAL = range(6)

PFF_OK = 0
(PFF_ERR_INVALID_ARG, PFF_ERR_OOM, PFF_ERR_CUDA, PFF_ERR_NAN, PFF_ERR_NOT_CONVERGED, PFF_ERR_BREAKDOWN,
 PFF_ERR_NO_STATE, PFF_ERR_TOO_LARGE, PFF_ERR_UNAVAILABLE) = range(-1, -10, -1)


class PFFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("n_cells_1d", ctypes.c_int),
                ("coarse_min", ctypes.c_int), ("split", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("mu", ctypes.c_double), ("gc", ctypes.c_double),
                ("eps", ctypes.c_double), ("kappa", ctypes.c_double), ("as_c", ctypes.c_double),
                ("mg_precision", ctypes.c_int), ("cheb_degree", ctypes.c_int),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double), ("eig_iters", ctypes.c_int),
                ("eig_seed", ctypes.c_ulonglong), ("gmres_restart", ctypes.c_int),
                ("gmres_max_iters", ctypes.c_int), ("lin_rtol", ctypes.c_double), ("fp64_mode", ctypes.c_int),
                ("coarse_precision", ctypes.c_int), ("slit_cut", ctypes.c_int),
                ("fp32_tangent", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("res_norm", ctypes.c_double), ("gmres_rel", ctypes.c_double), ("gmres_iters", ctypes.c_int),
                ("n_active", ctypes.c_int), ("n_changed", ctypes.c_int), ("status", ctypes.c_int),
                ("t_residual_ms", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_LIB = None

_P, _I, _D, _LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
_SIGS = {
    "pff_default_params": (None, [ctypes.POINTER(Params)]),
    "pff_setup_mesh": (_I, [ctypes.POINTER(_P), ctypes.POINTER(Params), _P]),
    "pff_destroy": (None, [_P]),
    "pff_sizes": (_I, [_P, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_I)]),
    "pff_level_sizes": (_I, [_P, _I, ctypes.POINTER(_LL), ctypes.POINTER(_I)]),
    "pff_node_flags": (_I, [_P, _I, _P]),
    "pff_set_state": (_I, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "pff_get_state": (_I, [_P, _P]),
    "pff_get_active": (_I, [_P, _P]),
    "pff_apply_jacobian": (_I, [_P, _I, _P, _P, _I, _I]),
    "pff_residual": (_I, [_P, _P]),
    "pff_reaction_force": (_I, [_P, ctypes.POINTER(_D)]),
    "pff_set_load_component": (_I, [_P, _I]),
    "pff_memory": (_I, [_P, _P, ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_LL), ctypes.POINTER(_LL)]),
    "pff_get_history": (_I, [_P, _P, _P, ctypes.POINTER(_I)]),
    "pff_csr_assemble": (_I, [_P, ctypes.POINTER(_LL)]),
    "pff_csr_spmv": (_I, [_P, _P, _P]),
    "pff_csr_spmv_available": (_I, []),
    "pff_csr_export": (_I, [_P, _P, _P, _P]),
    "pff_csr_pattern": (_I, [_I, _I, _I, _P, _P, _P, ctypes.POINTER(_LL)]),
    "pff_csr_probe_targets": (_I, [_I, _I, _I, _I, _I, _P]),
    "pff_set_history": (_I, [_P, _P, _P, _I]),
    "pff_diagonal": (_I, [_P, _I, _P, _I]),
    "pff_lambda_max": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "pff_level_state": (_I, [_P, _I, _P]),
    "pff_prolongate": (_I, [_P, _I, _P, _P, _I]),
    "pff_restrict": (_I, [_P, _I, _P, _P, _I]),
    "pff_smooth": (_I, [_P, _I, _P, _P, _I]),
    "pff_coarse_solve": (_I, [_P, _P, _P]),
    "pff_vcycle": (_I, [_P, _P, _P]),
    "pff_solve_linear": (_I, [_P, _P, _P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    "pff_solve_newton_step": (_I, [_P, _P, ctypes.POINTER(Report)]),
    "pff_solve_pdas": (_I, [_P, _I, _D, _P, ctypes.POINTER(Report), ctypes.POINTER(_I)]),
    "pff_solve_load_step": (_I, [_P, _D, _I, _D, ctypes.POINTER(Report), ctypes.POINTER(_I)]),
    "pff_param_grad": (_I, [_P, _P, _P, _P, _P]),
    "pff_param_grad_noalloc": (_I, [_P, _P, _P, _P, _P]),
    "pff_strerror": (ctypes.c_char_p, [_I]),
    "pff_profile": (_I, [_P, _I]),
    "pff_launch_count": (_LL, []),
    "pff_profile_result": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
}


def library_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libpff.so")


def load_library(build_if_missing=True):
    """Loads libpff.so (building it in-tree if it is missing); raises if that fails."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libpff.so is not built (%s); run paper_2005_00331_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, what):
    if status != 0:
        msg = load_library().pff_strerror(status).decode()
        raise PFFError(status, "%s failed: %s (%d)" % (what, msg, status))


def _ptr(t, dtype=torch.float64, numel=None):
    if t is None:
        return None
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise ValueError("expected a contiguous CUDA tensor of %s, got %s %s" % (dtype, t.dtype, t.device))
    if numel is not None and t.numel() != numel:
        raise ValueError("expected %d entries, got %d" % (numel, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def launch_count():
    """Kernels launched by libpff so far in this process."""
    return int(load_library().pff_launch_count())


def default_params(**kw):
    p = Params()
    load_library().pff_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lambda" else k, v)
    return p


class Context:
    """Owns one pff_ctx: the mesh hierarchy of one problem and its Newton state."""

    def __init__(self, params, stream=None):
        lib = load_library()
        self._lib = lib
        self.params = params
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.device = self.stream.device
        h = ctypes.c_void_p()
        _check(lib.pff_setup_mesh(ctypes.byref(h), ctypes.byref(params), ctypes.c_void_p(self.stream.cuda_stream)),
               "pff_setup_mesh")
        self._h = h
        nd, nn, nl = _LL(), _LL(), _I()
        _check(lib.pff_sizes(h, ctypes.byref(nd), ctypes.byref(nn), ctypes.byref(nl)), "pff_sizes")
        self.n_dofs, self.n_nodes, self.n_levels = nd.value, nn.value, nl.value
        self.dim = params.dim
        self.csr_nnz = 0

    def close(self):
        """Destroys the library context (pff_destroy); the object is unusable afterwards."""
        if getattr(self, "_h", None):
            self._lib.pff_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def level_sizes(self, level):
        """(n_nodes, n_cells_1d) of multigrid level `level` (0 = finest)."""
        nn, N = _LL(), _I()
        _check(self._lib.pff_level_sizes(self._h, level, ctypes.byref(nn), ctypes.byref(N)), "pff_level_sizes")
        return nn.value, N.value

    def _dev(self):
        """The device of the context's stream (where the library allocated everything)."""
        return self.device

    def node_flags(self, level=0):
        """Node flags of a level (pff_node_flags): bit f = DoF of component f masked, plus PFF_FLAG_*."""
        nn, _ = self.level_sizes(level)
        out = torch.empty(nn, dtype=torch.uint8, device=self._dev())
        _check(self._lib.pff_node_flags(self._h, level, _ptr(out, torch.uint8)), "pff_node_flags")
        return out

    def set_state(self, U, phi_old, phi_tilde=None, active=None, gc_field=None, lambda_field=None, mu_field=None):
        """Sets the Newton state (pff_set_state): U in the DoF layout, phi_old, phi~ (default phi_old),
        the active set (uint8 per node; None = computed by the rule of Alg. 1) and optional nodal fields."""
        nn = self.n_nodes
        _check(self._lib.pff_set_state(self._h, _ptr(U, numel=self.n_dofs), _ptr(phi_old, numel=nn),
                                       _ptr(phi_tilde, numel=nn), _ptr(active, torch.uint8, nn),
                                       _ptr(gc_field, numel=nn), _ptr(lambda_field, numel=nn),
                                       _ptr(mu_field, numel=nn)), "pff_set_state")

    def get_state(self):
        """Current state U (a new device tensor)."""
        out = torch.empty(self.n_dofs, dtype=torch.float64, device=self._dev())
        _check(self._lib.pff_get_state(self._h, _ptr(out)), "pff_get_state")
        return out

    def get_active(self):
        """Current active set, one byte per node (1 = active)."""
        out = torch.empty(self.n_nodes, dtype=torch.uint8, device=self._dev())
        _check(self._lib.pff_get_active(self._h, _ptr(out, torch.uint8)), "pff_get_active")
        return out

    def _level_nd(self, level):
        return (self.dim + 1) * self.level_sizes(level)[0]

    def apply_jacobian(self, x, y=None, level=0, mode=PFF_MODE_FULL, precision=None):
        """y = G x on `level` (pff_apply_jacobian); precision from x's dtype unless given, mode =
        PFF_MODE_* | PFF_MASK_*."""
        prec = precision or (32 if x.dtype == torch.float32 else 64)
        dt = torch.float32 if prec == 32 else torch.float64
        nd = self._level_nd(level)
        if y is None:
            y = torch.empty(nd, dtype=dt, device=x.device)
        _check(self._lib.pff_apply_jacobian(self._h, level, _ptr(x, dt, nd), _ptr(y, dt, nd), prec, mode),
               "pff_apply_jacobian")
        return y

    def residual(self, r=None):
        """r = R(U) of Eq. (residual), FP64, Dirichlet rows 0 (pff_residual)."""
        if r is None:
            r = torch.empty(self.n_dofs, dtype=torch.float64, device=self._dev())
        _check(self._lib.pff_residual(self._h, _ptr(r, numel=self.n_dofs)), "pff_residual")
        return r

    def diagonal(self, level=0, precision=64):
        """Jacobi diagonal diag(G_uu, G_phiphi) of a level, masked rows 1 (pff_diagonal)."""
        dt = torch.float32 if precision == 32 else torch.float64
        out = torch.empty(self._level_nd(level), dtype=dt, device=self._dev())
        _check(self._lib.pff_diagonal(self._h, level, _ptr(out, dt), precision), "pff_diagonal")
        return out

    def lambda_max(self, level=0):
        """[lambda_max(D^-1 G_uu), lambda_max(D^-1 G_phiphi)] of a level (CG-Lanczos estimate)."""
        arr = (_D * 2)()
        _check(self._lib.pff_lambda_max(self._h, level, arr), "pff_lambda_max")
        return [arr[0], arr[1]]

    def level_state(self, level):
        """The state carried to a coarse level (pff_level_state)."""
        out = torch.empty(self._level_nd(level), dtype=torch.float64, device=self._dev())
        _check(self._lib.pff_level_state(self._h, level, _ptr(out)), "pff_level_state")
        return out

    def prolongate(self, level, xc, precision=64):
        """Prolongation from level + 1 to `level` (pff_prolongate)."""
        dt = torch.float32 if precision == 32 else torch.float64
        y = torch.empty(self._level_nd(level), dtype=dt, device=xc.device)
        _check(self._lib.pff_prolongate(self._h, level, _ptr(xc, dt, self._level_nd(level + 1)), _ptr(y, dt),
                                        precision), "pff_prolongate")
        return y

    def restrict(self, level, xf, precision=64):
        """Restriction from `level` to level + 1, the transpose of the prolongation (pff_restrict)."""
        dt = torch.float32 if precision == 32 else torch.float64
        y = torch.empty(self._level_nd(level + 1), dtype=dt, device=xf.device)
        _check(self._lib.pff_restrict(self._h, level, _ptr(xf, dt, self._level_nd(level)), _ptr(y, dt), precision),
               "pff_restrict")
        return y

    def smooth(self, level, f, precision=64):
        """One block-diagonal Chebyshev-Jacobi smoothing of f from zero on a level (pff_smooth)."""
        dt = torch.float32 if precision == 32 else torch.float64
        x = torch.empty(self._level_nd(level), dtype=dt, device=f.device)
        _check(self._lib.pff_smooth(self._h, level, _ptr(f, dt, self._level_nd(level)), _ptr(x, dt), precision),
               "pff_smooth")
        return x

    def coarse_solve(self, r):
        """Exact block forward substitution on the coarsest level (pff_coarse_solve)."""
        z = torch.empty_like(r)
        _check(self._lib.pff_coarse_solve(self._h, _ptr(r, numel=self._level_nd(self.n_levels - 1)), _ptr(z)),
               "pff_coarse_solve")
        return z

    def vcycle(self, r, z=None):
        """z = V-cycle applied to r (pff_vcycle), the preconditioner of the linear solve."""
        z = torch.empty_like(r) if z is None else z
        _check(self._lib.pff_vcycle(self._h, _ptr(r, numel=self.n_dofs), _ptr(z, numel=self.n_dofs)), "pff_vcycle")
        return z

    def solve_linear(self, b, x=None, check=True):
        """FGMRES with the V-cycle on G x = b (pff_solve_linear); returns (x, iterations, relative residual)."""
        x = torch.empty_like(b) if x is None else x
        its, rel = _I(), _D()
        st = self._lib.pff_solve_linear(self._h, _ptr(b, numel=self.n_dofs), _ptr(x, numel=self.n_dofs),
                                        ctypes.byref(its), ctypes.byref(rel))
        if check:
            _check(st, "pff_solve_linear")
        return x, its.value, rel.value

    def solve_newton_step(self, U_out=None, check=True):
        """One step of Alg. 1 (pff_solve_newton_step); returns its report as a dict."""
        rep = Report()
        st = self._lib.pff_solve_newton_step(self._h, _ptr(U_out, numel=self.n_dofs), ctypes.byref(rep))
        if check:
            _check(st, "pff_solve_newton_step")
        return rep.as_dict()

    def param_grad_noalloc(self, g_gc, g_lambda, g_mu, v):
        """pff_param_grad_noalloc: like param_grad, but the library allocates nothing; the caller passes
        the three output tensors (one value per node each)."""
        _check(self._lib.pff_param_grad_noalloc(self._h, _ptr(v, numel=self.n_dofs), _ptr(g_gc, numel=self.n_nodes),
                                                _ptr(g_lambda, numel=self.n_nodes), _ptr(g_mu, numel=self.n_nodes)),
               "pff_param_grad_noalloc")
        return g_gc, g_lambda, g_mu

    def profile(self, family):
        """Starts timing one kernel family (PFF_PROF_*); 0 switches it off."""
        _check(self._lib.pff_profile(self._h, family), "pff_profile")

    def profile_result(self):
        """(launches, total ms) of the timed kernel family since pff_profile (synchronises)."""
        n, ms = _I(), _D()
        _check(self._lib.pff_profile_result(self._h, ctypes.byref(n), ctypes.byref(ms)), "pff_profile_result")
        return n.value, ms.value

    def solve_pdas(self, max_iters=30, newton_rtol=1e-8, U_out=None, check=True, log=None):
        """Alg. 1 repeated until the active set settles and ||R~|| <= newton_rtol ||R~_0||. With `log`
        (a text file), one JSON line per Newton step (see report_lines) is written to it."""
        reps = (Report * max_iters)()
        n = _I()
        st = self._lib.pff_solve_pdas(self._h, max_iters, newton_rtol, _ptr(U_out, numel=self.n_dofs), reps,
                                      ctypes.byref(n))
        out = [reps[i].as_dict() for i in range(n.value)]
        if log is not None:
            self._log(log, out, loop_status=st)
        if check:
            _check(st, "pff_solve_pdas")
        return st, out

    def solve_load_step(self, load, max_iters=30, newton_rtol=1e-8, check=True, log=None):
        """One quasi-static load step (top displacement `load`, phi~ extrapolated, Alg. 1 to tolerance).
        With `log` (a text file), one JSON line per Newton step, with the load and the force on the top
        face after the step."""
        reps = (Report * max_iters)()
        n = _I()
        st = self._lib.pff_solve_load_step(self._h, load, max_iters, newton_rtol, reps, ctypes.byref(n))
        out = [reps[i].as_dict() for i in range(n.value)]
        if log is not None:
            self._log(log, out, loop_status=st, load=load, reaction_force=self.reaction_force())
        if check:
            _check(st, "pff_solve_load_step")
        return st, out

    def _log(self, fh, reports, **fields):
        mem = self.memory()
        for line in report_lines(reports, device_bytes=mem["total"], level_bytes=mem["levels"], **fields):
            fh.write(line + "\n")
        fh.flush()

    def memory(self):
        """Device bytes the context holds (pff_memory): {"levels": [...], "krylov", "coarse", "other", "total"}."""
        lv = (_LL * self.n_levels)()
        k, c, o, t = _LL(), _LL(), _LL(), _LL()
        _check(self._lib.pff_memory(self._h, lv, ctypes.byref(k), ctypes.byref(c), ctypes.byref(o), ctypes.byref(t)),
               "pff_memory")
        return {"levels": list(lv), "krylov": k.value, "coarse": c.value, "other": o.value, "total": t.value}

    def set_load_component(self, comp):
        """Loaded displacement component of the load steps and the reaction force: dim - 1 (tension,
        the default) or 0 (shear test)."""
        _check(self._lib.pff_set_load_component(self._h, comp), "pff_set_load_component")

    def reaction_force(self):
        """Force on the loaded top face at the current state (pff_reaction_force), a Python float."""
        f = _D()
        _check(self._lib.pff_reaction_force(self._h, ctypes.byref(f)), "pff_reaction_force")
        return f.value

    def get_history(self):
        """(n_hist, phi1, phi2): the phase fields of the last two converged load steps (None where unknown)."""
        nn = self.n_nodes
        phi1 = torch.empty(nn, dtype=torch.float64, device=self._dev())
        phi2 = torch.empty(nn, dtype=torch.float64, device=self._dev())
        n = _I()
        _check(self._lib.pff_get_history(self._h, _ptr(phi1), _ptr(phi2), ctypes.byref(n)), "pff_get_history")
        return n.value, (phi1 if n.value >= 1 else None), (phi2 if n.value >= 2 else None)

    def set_history(self, phi1=None, phi2=None):
        """Installs the load-step history after set_state (phi2 only together with phi1)."""
        if phi2 is not None and phi1 is None:
            raise ValueError("phi2 needs phi1")
        n = 0 if phi1 is None else (1 if phi2 is None else 2)
        nn = self.n_nodes
        _check(self._lib.pff_set_history(self._h, _ptr(phi1, numel=nn), _ptr(phi2, numel=nn), n),
               "pff_set_history")

    def checkpoint(self, load=float("nan")):
        """Host copy of what the next load step reads (state and phase-field history), as a
        ``checkpoint.Checkpoint``; ``load`` records the last converged top displacement."""
        from . import checkpoint as ck
        n, phi1, phi2 = self.get_history()
        host = (lambda t: t.cpu().numpy() if t is not None else None)
        return ck.Checkpoint(self.params.dim, self.params.degree, self.params.n_cells_1d, float(load),
                             self.get_state().cpu().numpy(), n, host(phi1), host(phi2), self.params.slit_cut)

    def resume(self, ckpt, gc_field=None, lambda_field=None, mu_field=None):
        """Restores a checkpoint into this context (same mesh): set_state with phi_old = the last
        converged phase field (the state's own phase field when no step has converged), then the
        history. The next solve_load_step continues the checkpointed run."""
        ckpt.check_mesh(self.params.dim, self.params.degree, self.params.n_cells_1d, self.params.slit_cut)
        dev = self._dev()
        dvec = (lambda a: torch.from_numpy(a).to(device=dev, dtype=torch.float64).contiguous())
        U = dvec(ckpt.U)
        phi1 = dvec(ckpt.phi1) if ckpt.n_hist >= 1 else None
        phi2 = dvec(ckpt.phi2) if ckpt.n_hist >= 2 else None
        phi_old = phi1 if phi1 is not None else U[self.params.dim * self.n_nodes:].contiguous()
        self.set_state(U, phi_old, None, None, gc_field, lambda_field, mu_field)
        self.set_history(phi1, phi2)

    def csr_assemble(self):
        """Assembles the masked finest-level Jacobian into the context's CSR matrix; returns nnz."""
        nnz = _LL()
        _check(self._lib.pff_csr_assemble(self._h, ctypes.byref(nnz)), "pff_csr_assemble")
        self.csr_nnz = nnz.value
        return nnz.value

    def csr_spmv(self, x, y=None):
        """y = A x with the assembled matrix (cuSPARSE)."""
        if y is None:
            y = torch.empty(self.n_dofs, dtype=torch.float64, device=x.device)
        _check(self._lib.pff_csr_spmv(self._h, _ptr(x, numel=self.n_dofs), _ptr(y, numel=self.n_dofs)),
               "pff_csr_spmv")
        return y

    def csr_export(self):
        """(rowptr, col, val) of the assembled matrix as device tensors (int32, int32, float64)."""
        dev = self._dev()
        rowptr = torch.empty(self.n_dofs + 1, dtype=torch.int32, device=dev)
        col = torch.empty(self.csr_nnz, dtype=torch.int32, device=dev)
        val = torch.empty(self.csr_nnz, dtype=torch.float64, device=dev)
        _check(self._lib.pff_csr_export(self._h, _ptr(rowptr, torch.int32), _ptr(col, torch.int32), _ptr(val)),
               "pff_csr_export")
        return rowptr, col, val

    def param_grad(self, v):
        """(dR/dG_c)^T v, (dR/dlambda)^T v, (dR/dmu)^T v as nodal device tensors (pff_param_grad)."""
        outs = [torch.empty(self.n_nodes, dtype=torch.float64, device=v.device) for _ in range(3)]
        _check(self._lib.pff_param_grad(self._h, _ptr(v, numel=self.n_dofs), *[_ptr(o) for o in outs]),
               "pff_param_grad")
        return outs


def report_lines(reports, **fields):
    """JSON lines, one per Newton step: the step's number and report (||R~||, |A|, active-set changes,
    FGMRES iterations and relative residual, status, milliseconds per phase) with `fields` added to
    each line (e.g. the load, the loop's status, device bytes per level; a step's own keys win)."""
    import json
    return [json.dumps(dict(fields, newton_step=k, **r)) for k, r in enumerate(reports)]


def csr_pattern(dim, degree, n_cells_1d, flags):
    """Host-only pattern of the assembled comparator matrix (pff_csr_pattern) for host node flags
    (a uint8 numpy array, one byte per node): returns (rowptr, col) as int32 numpy arrays."""
    import numpy as np
    lib = load_library()
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    if fl.size != (degree * n_cells_1d + 1) ** dim:
        raise ValueError("expected %d node flags, got %d" % ((degree * n_cells_1d + 1) ** dim, fl.size))
    fp = fl.ctypes.data_as(ctypes.c_void_p)
    nnz = _LL()
    _check(lib.pff_csr_pattern(dim, degree, n_cells_1d, fp, None, None, ctypes.byref(nnz)), "pff_csr_pattern")
    rowptr = np.empty((dim + 1) * fl.size + 1, dtype=np.int32)
    col = np.empty(nnz.value, dtype=np.int32)
    _check(lib.pff_csr_pattern(dim, degree, n_cells_1d, fp, rowptr.ctypes.data_as(ctypes.c_void_p),
                               col.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nnz)), "pff_csr_pattern")
    return rowptr, col


def csr_probe_targets(dim, degree, n_cells_1d, f, color):
    """Host-only probing plan of the comparator assembly (pff_csr_probe_targets): for each row, the
    column that the probe (component f, colour) fills, or -1; an int64 numpy array."""
    import numpy as np
    out = np.empty((dim + 1) * (degree * n_cells_1d + 1) ** dim, dtype=np.int64)
    _check(load_library().pff_csr_probe_targets(dim, degree, n_cells_1d, f, color,
                                                out.ctypes.data_as(ctypes.c_void_p)), "pff_csr_probe_targets")
    return out


def setup_mesh(dim=2, degree=1, n_cells_1d=32, stream=None, **kw):
    """Creates a Context (pff_setup_mesh) with the library defaults overridden by ``kw``."""
    p = default_params(dim=dim, degree=degree, n_cells_1d=n_cells_1d, **kw)
    return Context(p, stream)


class ResidualFunction(torch.autograd.Function):
    """R(U; G_c, lambda, mu) of Eq. (residual) with Dirichlet rows 0, differentiable in U and in the
    nodal material fields. Backward: dR/dU^T v is the transpose Jacobian apply with the Dirichlet rows
    of v removed (PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT); dR/dfield^T v comes from pff_param_grad.
    phi_old and phi~ are constants (G is the derivative with phi~ frozen)."""

    @staticmethod
    def forward(fctx, ctx, U, phi_old, phi_tilde, gc_field, lambda_field, mu_field):
        active = torch.zeros(ctx.n_nodes, dtype=torch.uint8, device=U.device)
        ctx.set_state(U.detach().contiguous(), phi_old, phi_tilde, active, gc_field.detach().contiguous(),
                      lambda_field.detach().contiguous(), mu_field.detach().contiguous())
        fctx.ctx = ctx
        fctx.save_for_backward(U, phi_old, phi_tilde, gc_field, lambda_field, mu_field, active)
        return ctx.residual()

    @staticmethod
    def backward(fctx, v):
        U, phi_old, phi_tilde, gc, lam, mu, active = fctx.saved_tensors
        ctx = fctx.ctx
        ctx.set_state(U.detach().contiguous(), phi_old, phi_tilde, active, gc.detach().contiguous(),
                      lam.detach().contiguous(), mu.detach().contiguous())
        v = v.contiguous()
        gU = ctx.apply_jacobian(v, mode=PFF_MODE_TRANSPOSE | PFF_MASK_ADJOINT)
        g_gc, g_lam, g_mu = ctx.param_grad(v)
        return None, gU, None, None, g_gc, g_lam, g_mu
