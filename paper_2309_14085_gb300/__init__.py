"""GB300 (sm_103a) H2* fast matrix-vector product -- Python binding.

Thin ctypes binding over the C ABI declared in ``include/h2star.h``.  It only
marshals arguments: the hierarchical construction runs in the library's C++
host code, and every step of the matrix-vector product runs in its CUDA
kernels.  PyTorch is used for device memory and streams only.  There is no
CPU fallback: if ``libh2star.so`` is missing, every call raises.

    from paper_2309_14085_gb300 import H2Matrix
    A = H2Matrix(points, "log2d", leaf_size=64, tol=1e-8)       # host build + upload
    y = A.matvec(x)        # x: torch float64 CUDA tensor (N,) or (N, nrhs)
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libh2star.so")

KERNELS = {"log2d": 0, "invr": 1, "imq": 2, "matern12": 3}
VARIANTS = {"h2star": 0, "h2plush": 1, "h2sqrt": 2, "h2star_t": 3, "h2sqrt_t": 4, "h2star_b": 5}
STORAGE = {"f64": 0, "f32": 1, "df64": 2, "bf16": 3}
NEAR = {None: 0, "fly": 1, "stored": 2}
#: M2L coupling blocks: stored (formed on the host), evaluated in each product
#: from the pivot coordinates (fp32 only), or stored and formed on the device
M2L = {None: 0, "stored": 0, "fly": 1, "device": 2}
#: where the pivot search runs: by default the device for 1/r and the IMQ unless
#: host_only (the host for log r and exp(-r)), or forced
PIVOTS = {None: 0, "device": 1, "host": 2}
STAGES = ("gather", "p2m", "m2m", "m2l", "l2l", "leaf", "lowrank", "scatter")
EXPORTED = ("h2_build", "h2_convert", "h2_release_host", "h2_matvec", "h2_gmres", "h2_info", "h2_get_pivots", "h2_tree_order",
            "h2_profile", "h2_stage_times", "h2_last_error", "h2_destroy", "h2_batch_create",
            "h2_batch_matvec", "h2_batch_info", "h2_batch_destroy", "h2_server_create",
            "h2_server_submit", "h2_server_wait", "h2_server_stats_get", "h2_server_destroy",
            "h2_inject_wait_expiry", "h2_save", "h2_load")


class BuildOpts(ctypes.Structure):
    _fields_ = [("eps_far", ctypes.c_double), ("eps_ver", ctypes.c_double),
                ("storage", ctypes.c_int), ("kappa", ctypes.c_int),
                ("use_domain", ctypes.c_int), ("domain_lo", ctypes.c_double * 3),
                ("domain_side", ctypes.c_double), ("threads", ctypes.c_int),
                ("host_only", ctypes.c_int), ("kparam", ctypes.c_double),
                ("near_mode", ctypes.c_int), ("tensor_cores", ctypes.c_int),
                ("m2l_mode", ctypes.c_int), ("pivots", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("d", ctypes.c_int), ("kappa", ctypes.c_int),
                ("kernel", ctypes.c_int), ("variant", ctypes.c_int), ("storage", ctypes.c_int),
                ("nbases", ctypes.c_int),
                ("rank_min", (ctypes.c_int * 32) * 2), ("rank_max", (ctypes.c_int * 32) * 2),
                ("rank_avg", (ctypes.c_double * 32) * 2),
                ("m2l_pairs", ctypes.c_int64 * 2), ("near_pairs", ctypes.c_int64),
                ("near_evals", ctypes.c_int64), ("lowrank_pairs", ctypes.c_int64),
                ("bytes_basis", ctypes.c_int64), ("bytes_transfer", ctypes.c_int64),
                ("bytes_m2l", ctypes.c_int64), ("m2l_src_coeffs", ctypes.c_int64),
                ("m2l_dst_coeffs", ctypes.c_int64), ("vlen", ctypes.c_int64),
                ("bytes_leaf_rows", ctypes.c_int64), ("leaf_src_coeffs", ctypes.c_int64),
                ("near_stored", ctypes.c_int), ("rw_m2l", ctypes.c_int), ("rw_leaf", ctypes.c_int),
                ("bytes_lowrank", ctypes.c_int64),
                ("bytes_device", ctypes.c_int64), ("alg_bytes_per_rhs", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("tc_blocks", ctypes.c_int * 3),
                ("tc_occupancy", ctypes.c_int * 3), ("m2l_fly", ctypes.c_int),
                ("m2l_entries", ctypes.c_int64), ("pivot_problems_device", ctypes.c_int64),
                ("pivot_problems_host", ctypes.c_int64), ("pivot_seconds", ctypes.c_double)]


class GmresStats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int),
                ("restarts", ctypes.c_int), ("refinements", ctypes.c_int),
                ("matvecs", ctypes.c_int64), ("matvecs_residual", ctypes.c_int64),
                ("rel_residual", ctypes.c_double), ("rel_residual_est", ctypes.c_double),
                ("seconds", ctypes.c_double), ("fallback", ctypes.c_int), ("pad_", ctypes.c_int)]


class BatchStats(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_int), ("virtual_instances", ctypes.c_int),
                ("points_times_rhs", ctypes.c_int64), ("launches_per_product", ctypes.c_int64),
                ("m2m_steps", ctypes.c_int), ("l2l_steps", ctypes.c_int),
                ("m2l_tasks", ctypes.c_int64), ("leaf_tasks", ctypes.c_int64),
                ("bytes_device", ctypes.c_int64), ("bytes_ops", ctypes.c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("workspace_bytes", ctypes.c_int64), ("restart", ctypes.c_int),
                ("max_active", ctypes.c_int), ("inner_policy", ctypes.c_int), ("pad_", ctypes.c_int)]


class ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "submitted", "admitted", "completed", "queued", "active", "max_active", "ticks",
        "products", "product_columns", "workspace_bytes")]


class RequestStats(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iterations", ctypes.c_int),
                ("restarts", ctypes.c_int), ("op", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("queue_seconds", ctypes.c_double), ("latency_seconds", ctypes.c_double)]


#: Status codes of the C ABI (the H2_OK / H2_E_* defines of h2star.h).
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED",
          -5: "UNSUPPORTED", -6: "NO_DEVICE", -7: "TIMEOUT"}


class H2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"h2 error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code
        self.status = STATUS.get(code)


_lib = None


def lib():
    """Load libh2star.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2309_14085_gb300.build_lib`")
        L = ctypes.CDLL(LIB_PATH)
        c_i64, c_int, c_vp, c_dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.c_double
        L.h2_build.argtypes = [c_vp, c_i64, c_int, c_int, c_int, c_dbl, c_int,
                               ctypes.POINTER(BuildOpts), ctypes.POINTER(c_vp)]
        L.h2_matvec.argtypes = [c_vp, c_vp, c_i64, c_vp, c_i64, c_int, c_vp]
        L.h2_info.argtypes = [c_vp, ctypes.POINTER(Stats)]
        L.h2_gmres.argtypes = [c_vp, c_vp, c_dbl, c_dbl, c_vp, c_vp, c_dbl, c_int, c_int,
                               ctypes.POINTER(GmresStats), c_vp]
        L.h2_get_pivots.argtypes = [c_vp, c_int, c_int, c_i64, c_vp, c_vp, c_i64,
                                    ctypes.POINTER(c_int)]
        L.h2_tree_order.argtypes = [c_vp, c_vp]
        L.h2_profile.argtypes = [c_vp, c_int]
        L.h2_stage_times.argtypes = [c_vp, c_vp, c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]
        L.h2_batch_create.argtypes = [c_vp, c_int, c_vp, ctypes.POINTER(c_vp)]
        L.h2_batch_matvec.argtypes = [c_vp, c_vp, c_vp, c_vp]
        L.h2_batch_info.argtypes = [c_vp, ctypes.POINTER(BatchStats)]
        L.h2_batch_destroy.argtypes = [c_vp]
        L.h2_batch_destroy.restype = None
        L.h2_convert.argtypes = [c_vp, c_int, ctypes.POINTER(c_vp)]
        L.h2_release_host.argtypes = [c_vp]
        L.h2_inject_wait_expiry.argtypes = [c_vp, c_i64, c_vp]
        L.h2_save.argtypes = [c_vp, ctypes.c_char_p]
        L.h2_load.argtypes = [ctypes.c_char_p, c_int, ctypes.POINTER(c_vp)]
        L.h2_server_create.argtypes = [c_vp, c_vp, c_int, ctypes.POINTER(ServerOpts),
                                       ctypes.POINTER(c_vp)]
        L.h2_server_submit.argtypes = [c_vp, c_int, c_dbl, c_dbl, c_vp, c_dbl, c_int,
                                       ctypes.POINTER(c_i64)]
        L.h2_server_wait.argtypes = [c_vp, c_i64, c_vp, ctypes.POINTER(RequestStats)]
        L.h2_server_stats_get.argtypes = [c_vp, ctypes.POINTER(ServerStats)]
        L.h2_server_destroy.argtypes = [c_vp]
        L.h2_server_destroy.restype = None
        L.h2_last_error.restype = ctypes.c_char_p
        L.h2_destroy.argtypes = [c_vp]
        L.h2_destroy.restype = None
        for name in EXPORTED:
            if name not in ("h2_last_error", "h2_destroy", "h2_batch_destroy", "h2_server_destroy"):
                getattr(L, name).restype = c_int
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise H2Error(rc, lib().h2_last_error().decode())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class H2Matrix:
    """A compressed kernel matrix K~ (H2*(b+t), (H2+H)* or H2_sqrt(d)(b)).

    `pivots`: where the ACA pivot search of the construction runs -- None (the
    device for 1/r and the IMQ unless host_only, else the host), "device" or
    "host"; the device search takes the host's decisions (h2_build_opts.pivots).
    """

    def __init__(self, points, kernel, leaf_size=64, tol=1e-8, variant="h2star", storage="f64",
                 eps_far=None, eps_ver=None, kappa=None, domain=None, threads=0,
                 host_only=False, kparam=None, near=None, tensor_cores=False, m2l=None,
                 pivots=None):
        P = np.ascontiguousarray(points, dtype=np.float64)
        if P.ndim != 2:
            raise ValueError("points must be N x d")
        self.N, self.d = P.shape
        self.kernel, self.variant, self.storage = kernel, variant, storage
        o = BuildOpts()
        o.eps_far = eps_far or 0.0
        o.eps_ver = eps_ver or 0.0
        o.storage = STORAGE[storage]
        o.kappa = -1 if kappa == "strict" else (kappa or 0)
        if domain is not None:
            lo, side = domain
            o.use_domain = 1
            for k in range(self.d):
                o.domain_lo[k] = float(lo[k])
            o.domain_side = float(side)
        o.threads = threads
        o.host_only = int(host_only)
        o.kparam = kparam or 0.0
        o.near_mode = NEAR[near]
        o.tensor_cores = int(tensor_cores)
        o.m2l_mode = M2L[m2l]
        o.pivots = PIVOTS[pivots]
        h = ctypes.c_void_p()
        _check(lib().h2_build(P.ctypes.data, self.N, self.d, KERNELS[kernel], leaf_size, tol,
                              VARIANTS[variant], ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def convert(self, storage):
        """A second device copy of this operator in another storage ("f64",
        "f32" or "df64"), without repeating the construction."""
        h = ctypes.c_void_p()
        _check(lib().h2_convert(self._h, STORAGE[storage], ctypes.byref(h)))
        m = H2Matrix.__new__(H2Matrix)
        m.N, m.d, m.kernel, m.variant, m.storage = self.N, self.d, self.kernel, self.variant, storage
        m._h = h
        return m

    def save(self, path):
        """Write the whole constructed representation to `path` (h2_save)."""
        _check(lib().h2_save(self._h, os.fsencode(path)))

    @classmethod
    def load(cls, path, host_only=False):
        """A matrix read from a file written by save(): host-only, or uploaded to
        the current CUDA device in the saved storage (h2_load)."""
        h = ctypes.c_void_p()
        _check(lib().h2_load(os.fsencode(path), int(host_only), ctypes.byref(h)))
        m = cls.__new__(cls)
        m._h = h
        st = m.info()
        inv = lambda table, v: next(k for k, x in table.items() if x == v)
        m.N, m.d = st["N"], st["d"]
        m.kernel = inv(KERNELS, st["kernel"])
        m.variant = inv(VARIANTS, st["variant"])
        m.storage = inv(STORAGE, st["storage"])
        return m

    def release_host(self):
        """Free the host copy of the operators (the device copy stays)."""
        _check(lib().h2_release_host(self._h))

    # -- the product ---------------------------------------------------------
    def matvec(self, X, out=None, stream=None):
        """Y = K~ X for a float64 CUDA tensor X of shape (N,) or (N, nrhs)."""
        import torch
        if X.dtype != torch.float64 or not X.is_cuda:
            raise ValueError("X must be a float64 CUDA tensor")
        vec = X.dim() == 1
        X2 = X.reshape(self.N, 1) if vec else X
        nrhs = X2.shape[1]
        Xc = X2 if (X2.stride(0) == 1 and (nrhs == 1 or X2.stride(1) >= self.N)) else \
            X2.t().contiguous().t()
        ldx = self.N if nrhs == 1 else Xc.stride(1)
        if out is None:
            Y = torch.empty((nrhs, self.N), dtype=torch.float64, device=X.device).t()
        else:
            Y = out.reshape(self.N, 1) if out.dim() == 1 else out
            if Y.stride(0) != 1:
                raise ValueError("out must be column-major")
        ldy = self.N if nrhs == 1 else Y.stride(1)
        _check(lib().h2_matvec(self._h, ctypes.c_void_p(Xc.data_ptr()), ldx,
                               ctypes.c_void_p(Y.data_ptr()), ldy, nrhs, _stream_ptr(stream)))
        if out is not None:
            return out
        return Y.reshape(self.N) if vec else Y

    def inject_wait_expiry(self, rounds=1 << 12, stream=None):
        """Run the expiry path of the tensor-core kernels' bounded waits (no GPU
        fault): afterwards every product on this matrix raises H2Error with
        status TIMEOUT.  Asynchronous on `stream`."""
        _check(lib().h2_inject_wait_expiry(self._h, rounds, _stream_ptr(stream)))

    # -- solves ------------------------------------------------------------------
    def gmres(self, b, shift=0.0, scale=1.0, rtol=1e-10, restart=100, maxit=1000,
              residual=None, out=None, stream=None):
        """x solving (shift I + scale K~) x = b (fp64 CUDA tensor b, shape (N,)).

        `residual`: optional second H2Matrix on the same points (e.g. fp64
        storage when this one is fp32) for mixed-precision iterative refinement.
        Returns (x, stats dict); stats["converged"] tells whether rtol was met."""
        import torch
        if b.dtype != torch.float64 or not b.is_cuda or b.dim() != 1 or b.shape[0] != self.N:
            raise ValueError("b must be a float64 CUDA vector of length N")
        b = b.contiguous()
        x = torch.empty_like(b) if out is None else out
        st = GmresStats()
        rc = lib().h2_gmres(self._h, residual._h if residual is not None else None, shift, scale,
                            ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), rtol,
                            restart, maxit, ctypes.byref(st), _stream_ptr(stream))
        if rc not in (0, -4):
            _check(rc)
        return x, {f[0]: getattr(st, f[0]) for f in GmresStats._fields_}

    # -- introspection -----------------------------------------------------------
    def info(self):
        st = Stats()
        _check(lib().h2_info(self._h, ctypes.byref(st)))
        out = {f[0]: getattr(st, f[0]) for f in Stats._fields_
               if f[0] not in ("rank_min", "rank_max", "rank_avg", "m2l_pairs", "tc_blocks",
                               "tc_occupancy")}
        out["m2l_pairs"] = list(st.m2l_pairs)
        out["tc_blocks"] = list(st.tc_blocks)
        out["tc_occupancy"] = list(st.tc_occupancy)
        out["ranks"] = [{l: (st.rank_min[b][l], round(st.rank_avg[b][l], 2), st.rank_max[b][l])
                         for l in range(st.kappa + 1) if st.rank_max[b][l] > 0}
                        for b in range(st.nbases)]
        return out

    def pivots(self, basis, level, box):
        """(t^{X,i}, s^{X,i}) as user point indices, in selection order."""
        cap = 4096
        ti = np.zeros(cap, dtype=np.int64)
        si = np.zeros(cap, dtype=np.int64)
        r = ctypes.c_int()
        _check(lib().h2_get_pivots(self._h, basis, level, box, ti.ctypes.data, si.ctypes.data,
                                   cap, ctypes.byref(r)))
        return ti[:r.value].copy(), si[:r.value].copy()

    def tree_order(self):
        perm = np.zeros(self.N, dtype=np.int64)
        _check(lib().h2_tree_order(self._h, perm.ctypes.data))
        return perm

    def profile(self, enable=True):
        _check(lib().h2_profile(self._h, int(enable)))

    def stage_times(self):
        """(ms per stage accumulated, pipeline runs timed, kernels launched)."""
        ms = np.zeros(8)
        calls, launches = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().h2_stage_times(self._h, ms.ctypes.data, 8, ctypes.byref(calls),
                                    ctypes.byref(launches)))
        return dict(zip(STAGES, ms.tolist())), calls.value, launches.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().h2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class H2Batch:
    """Many independent compressed matrices applied together: one captured
    CUDA graph of merged, level-synchronous launches per batched product."""

    def __init__(self, matrices, nrhs=None):
        self.matrices = list(matrices)
        n = len(self.matrices)
        self.nrhs = list(nrhs) if nrhs is not None else [1] * n
        hs = (ctypes.c_void_p * n)(*[m._h.value for m in self.matrices])
        nr = (ctypes.c_int * n)(*self.nrhs)
        h = ctypes.c_void_p()
        _check(lib().h2_batch_create(hs, n, nr, ctypes.byref(h)))
        self._h = h

    def info(self):
        st = BatchStats()
        _check(lib().h2_batch_info(self._h, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in BatchStats._fields_}

    def matvec(self, xs, outs=None, stream=None):
        """xs[i]: float64 CUDA tensor (N_i,) or (N_i, nrhs_i); returns the products."""
        import torch
        n = len(self.matrices)
        cols, outs2 = [], []
        for i, (m, x) in enumerate(zip(self.matrices, xs)):
            x2 = x.reshape(m.N, -1)
            if x2.shape[1] != self.nrhs[i] or x2.dtype != torch.float64 or not x2.is_cuda:
                raise ValueError(f"input {i} must be float64 CUDA with {self.nrhs[i]} columns")
            cols.append(x2.t().contiguous())            # (nrhs, N): column c contiguous
            outs2.append(torch.empty((self.nrhs[i], m.N), dtype=torch.float64, device=x.device)
                         if outs is None else outs[i])
        X = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cols])
        Y = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs2])
        _check(lib().h2_batch_matvec(self._h, X, Y, _stream_ptr(stream)))
        self._keep = (cols, outs2)
        return [o.t() if self.nrhs[i] > 1 else o.reshape(-1) for i, o in enumerate(outs2)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().h2_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class H2Server:
    """Continuous-batching solve server over resident geometries (H2Matrix on
    the device).  submit() queues a solve and returns at once; wait() blocks
    for its solution; requests that arrive while others run join the active
    set as workspace frees up."""

    def __init__(self, geometries, workspace_bytes=0, restart=50, max_active=16, residual=None,
                 inner_policy=0):
        """`residual`: None, or one H2Matrix per geometry (same points) whose
        operator computes the residual that starts every GMRES cycle, e.g. the
        fp64 source of fp32 geometries made by H2Matrix.convert("f32").
        `inner_policy`: 0 admits a request on the inner operator only if its
        measured error is below |shift| / 10; 1 always starts there."""
        self.geometries = list(geometries)
        self.residual = list(residual) if residual is not None else None
        n = len(self.geometries)
        hs = (ctypes.c_void_p * n)(*[g._h.value for g in self.geometries])
        rs = None
        if self.residual is not None:
            if len(self.residual) != n:
                raise ValueError("one residual matrix per geometry")
            rs = (ctypes.c_void_p * n)(*[g._h.value for g in self.residual])
        o = ServerOpts(workspace_bytes, restart, max_active, inner_policy, 0)
        h = ctypes.c_void_p()
        _check(lib().h2_server_create(hs, rs, n, ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def submit(self, geom, f, shift=0.0, scale=1.0, rtol=1e-8, maxit=1000):
        f = np.ascontiguousarray(f, dtype=np.float64)
        t = ctypes.c_int64()
        _check(lib().h2_server_submit(self._h, geom, shift, scale, f.ctypes.data, rtol, maxit,
                                      ctypes.byref(t)))
        return t.value

    def wait(self, ticket):
        """(x, stats) of a submitted request; stats["converged"] tells whether rtol was met."""
        # the ticket's geometry is not tracked here: the library copies N values
        st = RequestStats()
        x = np.zeros(max(g.N for g in self.geometries))
        rc = lib().h2_server_wait(self._h, ticket, x.ctypes.data, ctypes.byref(st))
        if rc not in (0, -4):
            _check(rc)
        return x, {f[0]: getattr(st, f[0]) for f in RequestStats._fields_}

    def stats(self):
        st = ServerStats()
        _check(lib().h2_server_stats_get(self._h, ctypes.byref(st)))
        return {f[0]: getattr(st, f[0]) for f in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().h2_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

