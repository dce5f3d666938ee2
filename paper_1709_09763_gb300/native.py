"""ctypes binding of libmls2mc.so: the C ABI of include/mls2mc.h, argument marshalling only.

Every computation happens inside the library's CUDA kernels. Loading fails loudly
when the library has not been built; there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmls2mc.so")

SMC_OK = 0
SMC_EINVAL = -1
SMC_ENOMEM = -2
SMC_ECUDA = -3
SMC_ENOCONV = -4
SMC_ESINGULAR = -5
SMC_ETIMEOUT = -6
SMC_FP64 = 0
SMC_MIXED = 1
SMC_FWD_FEM = 0
SMC_FWD_LINEAR = 1
SMC_COV_SEP_EXP = 0
SMC_COV_MATERN = 1
SMC_SRC_ONE = 0
SMC_SRC_NINE = 1
SMC_PROP_PCN = 0
SMC_PROP_RWM = 1
SMC_PROP_RWM_COV = 2
_COV = {"sep_exp": SMC_COV_SEP_EXP, "matern": SMC_COV_MATERN}
_SRC = {"one": SMC_SRC_ONE, "nine": SMC_SRC_NINE}
_PROP = {"pcn": SMC_PROP_PCN, "rwm": SMC_PROP_RWM, "rwm_cov": SMC_PROP_RWM_COV}
SMC_BC_DIRICHLET = 0
SMC_BC_FLOW_CELL = 1
_BC = {"dirichlet": SMC_BC_DIRICHLET, "flow_cell": SMC_BC_FLOW_CELL}
SMC_NOALLOC_MAX_PARTICLES = 65536

ERROR_NAMES = {0: "SMC_OK", -1: "SMC_EINVAL", -2: "SMC_ENOMEM", -3: "SMC_ECUDA", -4: "SMC_ENOCONV",
               -5: "SMC_ESINGULAR", -6: "SMC_ETIMEOUT"}

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class ProblemDesc(ctypes.Structure):
    _fields_ = [("n_levels", ctypes.c_int), ("inv_h", _ip), ("K", ctypes.c_int),
                ("corr_len", ctypes.c_double), ("variance", ctypes.c_double),
                ("n_obs", ctypes.c_int), ("obs_xy", _dp), ("y", _dp), ("sigma", ctypes.c_double),
                ("forward_kind", ctypes.c_int), ("linear_A", _dp), ("cov_kind", ctypes.c_int),
                ("source_kind", ctypes.c_int), ("bc_kind", ctypes.c_int)]


class SamplerOpts(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int), ("J_tilde", ctypes.c_int), ("n_mcmc", ctypes.c_int),
                ("tau_star", ctypes.c_double), ("tau_lu", ctypes.c_double), ("eps", ctypes.c_double),
                ("s_pcn", ctypes.c_double), ("precision", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("max_iter", ctypes.c_int), ("rtol", ctypes.c_double), ("surrogate", ctypes.c_int),
                ("surrogate_train_steps", ctypes.c_int), ("surrogate_batch", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("proposal", ctypes.c_int), ("tau_min", ctypes.c_double),
                ("accept_target", ctypes.c_double)]


class StageInfo(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("level", ctypes.c_int), ("beta", ctypes.c_double),
                ("zeta", ctypes.c_double), ("delta", ctypes.c_double), ("cv", ctypes.c_double),
                ("cv_lu", ctypes.c_double), ("log_z_inc", ctypes.c_double),
                ("accept_rate", ctypes.c_double), ("da_stage1_rate", ctypes.c_double),
                ("evals_per_level", ctypes.c_longlong * 8), ("n_bridge", ctypes.c_int), ("status", ctypes.c_int),
                ("n_unique", ctypes.c_int), ("pad", ctypes.c_int), ("step", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("evals_per_level", "pad")}
        d["evals_per_level"] = list(self.evals_per_level)
        d["kind"] = "ITU" if self.type == 0 else "LU"
        return d


_lib = None

# name -> (restype, argtypes); every function the header declares
SIGNATURES = {
    "smc_init": (ctypes.c_int, [ctypes.POINTER(ProblemDesc), ctypes.POINTER(SamplerOpts),
                                ctypes.POINTER(ctypes.c_void_p)]),
    "smc_destroy": (None, [ctypes.c_void_p]),
    "smc_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "smc_eval_likelihood": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]),
    "smc_eval_likelihood_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_void_p]),
    "smc_kl_table": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, _dp]),
    "smc_kl_table_host": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                         _dp, _dp]),
    "smc_sizes": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip, _ip, _ip]),
    "smc_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(StageInfo)]),
    "smc_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StageInfo)]),
    "smc_state": (ctypes.c_int, [ctypes.c_void_p, _ip, _dp, _dp, _ip, ctypes.POINTER(ctypes.c_longlong)]),
    "smc_surrogate_gate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, _dp, _dp]),
    "smc_path": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(StageInfo), _ip]),
    "smc_posterior_moments": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp]),
    "smc_get_particles": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "smc_set_particles": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "smc_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "smc_kernel_launches": (ctypes.c_longlong, []),
    "smc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_void_p]),
    "smc_set_block_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "smc_block_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip]),
    "smc_get_timing": (ctypes.c_int, [ctypes.c_void_p, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "smc_get_phase_timing": (ctypes.c_int, [ctypes.c_void_p, _dp]),
    "smc_tempering_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(StageInfo)]),
    "smc_bridging_update": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_int, ctypes.POINTER(StageInfo)]),
    "smc_next_increment": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_double, _dp]),
    "smc_systematic_resample": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _dp, ctypes.c_double, _ip]),
    "smc_philox_normals": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                                          ctypes.c_uint, _dp]),
    "smc_systematic_resample_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                                                       ctypes.c_void_p, ctypes.c_void_p]),
    "smc_surrogate_dims": (ctypes.c_int, [ctypes.c_void_p, _ip]),
    "smc_surrogate_add_pairs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp]),
    "smc_surrogate_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]),
    "smc_surrogate_predict": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]),
    "smc_surrogate_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "smc_surrogate_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_void_p,
                                           _dp]),
    "smc_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "smc_batch_eval": (ctypes.c_int, [ctypes.c_void_p, _ip, _ip, ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.c_void_p, ctypes.c_int]),
    "smc_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "smc_init_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ProblemDesc), ctypes.POINTER(SamplerOpts),
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "smc_batch_handle": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int]),
    "smc_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(StageInfo)]),
    "smc_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip]),
    "smc_batch_destroy": (None, [ctypes.c_void_p]),
    "smc_gemm_bf16": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "smc_philox_uniforms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_uint, _dp]),
}


def load():
    """Load libmls2mc.so (build it first with paper_1709_09763_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_1709_09763_gb300.build` "
                           "(the CUDA library is required; there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def bf16_bits(x):
    """Round-to-nearest-even BF16 bit patterns (uint16) of an FP32/FP64 array."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_value(bits):
    return (np.asarray(bits, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def gemm_bf16(A, B):
    """C = A . B^T on the tensor cores; A (M, K), B (N, K) are rounded to BF16 first."""
    lib = load()
    a = bf16_bits(A)
    b = bf16_bits(B)
    M, K = a.shape
    N = b.shape[0]
    C = np.empty((M, N), dtype=np.float32)
    rc = lib.smc_gemm_bf16(M, N, K, a.ctypes.data, b.ctypes.data, C.ctypes.data)
    if rc != SMC_OK:
        raise SmcError(rc, "smc_gemm_bf16")
    return C


def kl_table_host(cov, N, corr_len, variance, K):
    """KL table Psi [K][2 N^2] and eigenvalues [K] computed on the host (no handle, no GPU)."""
    lib = load()
    psi = np.empty((K, 2 * N * N))
    lam = np.empty(K)
    rc = lib.smc_kl_table_host(_COV[cov], N, corr_len, variance, K, _dptr(psi), _dptr(lam))
    if rc != SMC_OK:
        raise SmcError(rc, "smc_kl_table_host")
    return psi, lam


class Batch:
    """Independent problems evaluated together (persistent launch per level size, CUDA graph)."""

    def __init__(self, handles):
        self._lib = load()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        out = ctypes.c_void_p()
        rc = self._lib.smc_batch_create(len(self.handles), arr, ctypes.byref(out))
        if rc != SMC_OK:
            raise SmcError(rc, "smc_batch_create")
        self._b = out

    def eval(self, levels, counts, theta_ptrs, phi_ptrs, iters_ptrs=None, stream=None, use_graph=True):
        P = len(self.handles)
        lv = (ctypes.c_int * P)(*levels)
        cn = (ctypes.c_int * P)(*counts)
        th = (ctypes.c_void_p * P)(*theta_ptrs)
        ph = (ctypes.c_void_p * P)(*phi_ptrs)
        it = (ctypes.c_void_p * P)(*iters_ptrs) if iters_ptrs is not None else None
        rc = self._lib.smc_batch_eval(self._b, lv, cn, th, ph, it, stream, int(use_graph))
        if rc != SMC_OK:
            raise SmcError(rc, self._lib.smc_batch_last_error(self._b).decode())

    # ---- the batched sampler (every problem's next update in shared launches) ---------------
    def _check(self, rc, what):
        if rc != SMC_OK:
            raise SmcError(rc, f"{what}: {self._lib.smc_batch_last_error(self._b).decode()}")

    def step(self):
        """One importance-sampling update of every unfinished problem; returns their records."""
        P = len(self.handles)
        infos = (StageInfo * P)()
        self._check(self._lib.smc_batch_step(self._b, infos), "smc_batch_step")
        return [i.as_dict() for i in infos]

    def run(self, max_steps=0):
        """Steps until every problem is finished; returns the number of batched steps."""
        n = ctypes.c_int()
        self._check(self._lib.smc_batch_run(self._b, int(max_steps), ctypes.byref(n)), "smc_batch_run")
        return n.value

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            self._lib.smc_batch_destroy(self._b)
        self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def init_batch(problems):
    """smc_init_batch: a batch that owns one handle per problem; `problems` is a list of keyword
    dicts of Handle (inv_h, K, obs_xy, y, sigma and the options). The handles are available as
    batch.handles (views, destroyed with the batch)."""
    lib = load()
    P = len(problems)
    ds, os_, keep = (ProblemDesc * P)(), (SamplerOpts * P)(), []
    for i, kw in enumerate(problems):
        kw = dict(kw)
        d, o, k = _desc_opts(kw.pop("inv_h"), kw.pop("K"), kw.pop("obs_xy"), kw.pop("y"), kw.pop("sigma"), **kw)
        ds[i], os_[i] = d, o
        keep.append(k)
    out = ctypes.c_void_p()
    rc = lib.smc_init_batch(P, ds, os_, ctypes.byref(out))
    if rc != SMC_OK:
        raise SmcError(rc, "smc_init_batch")
    b = Batch.__new__(Batch)
    b._lib = lib
    b._b = out
    b.handles = [Handle.borrowed(lib.smc_batch_handle(out, p), b) for p in range(P)]
    return b


class SmcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _dptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _desc_opts(inv_h, K, obs_xy, y, sigma, corr_len=0.1, variance=1.0, J=0, J_tilde=100, n_mcmc=5, tau_star=1.0,
               tau_lu=None, eps=1e-6, s_pcn=0.2, precision=SMC_FP64, seed=0, max_iter=100, rtol=0.0, stream=None,
               linear_A=None, surrogate=0, surrogate_train_steps=0, surrogate_batch=0, cov="sep_exp",
               source="one", proposal="pcn", tau_min=0.0, bc="dirichlet", accept_target=0.0):
    """smc_problem_desc and smc_sampler_opts of the keyword form, and the arrays they point to."""
    inv_h = np.ascontiguousarray(inv_h, dtype=np.int32)
    obs = np.ascontiguousarray(obs_xy, dtype=np.float64).reshape(-1, 2)
    yy = np.ascontiguousarray(y, dtype=np.float64).ravel()
    A = None if linear_A is None else np.ascontiguousarray(linear_A, dtype=np.float64)
    d = ProblemDesc(len(inv_h), inv_h.ctypes.data_as(_ip), int(K), float(corr_len), float(variance), obs.shape[0],
                    _dptr(obs), _dptr(yy), float(sigma), SMC_FWD_LINEAR if A is not None else SMC_FWD_FEM, _dptr(A),
                    _COV[cov], _SRC[source], _BC[bc])
    o = SamplerOpts(int(J), int(J_tilde), int(n_mcmc), float(tau_star), float(tau_star if tau_lu is None else tau_lu),
                    float(eps), float(s_pcn), int(precision), int(seed), int(max_iter), float(rtol), int(surrogate),
                    int(surrogate_train_steps), int(surrogate_batch), stream, _PROP[proposal], float(tau_min),
                    float(accept_target))
    return d, o, (inv_h, obs, yy, A)


class Handle:
    """Owns one smc_handle. Arrays passed in are kept alive for the call's duration only."""

    def __init__(self, inv_h, K, obs_xy, y, sigma, **kw):
        lib = load()
        self._lib = lib
        d, o, self._keep = _desc_opts(inv_h, K, obs_xy, y, sigma, **kw)
        h = ctypes.c_void_p()
        rc = lib.smc_init(ctypes.byref(d), ctypes.byref(o), ctypes.byref(h))
        self._h = h
        if rc != SMC_OK:
            msg = lib.smc_last_error(h).decode() if h.value else "no handle"
            self.close()
            raise SmcError(rc, msg)
        K_, n_obs, nl, J_ = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        lib.smc_sizes(h, ctypes.byref(K_), ctypes.byref(n_obs), ctypes.byref(nl), ctypes.byref(J_))
        self.K, self.n_obs, self.n_levels, self.J = K_.value, n_obs.value, nl.value, J_.value

    @classmethod
    def borrowed(cls, ptr, owner):
        """A view of a handle that `owner` (a Batch made by init_batch) owns and destroys."""
        self = cls.__new__(cls)
        self._lib = load()
        self._h = ctypes.c_void_p(ptr)
        self._owner = owner
        K_, n_obs, nl, J_ = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._lib.smc_sizes(self._h, ctypes.byref(K_), ctypes.byref(n_obs), ctypes.byref(nl), ctypes.byref(J_))
        self.K, self.n_obs, self.n_levels, self.J = K_.value, n_obs.value, nl.value, J_.value
        return self

    def close(self):
        if getattr(self, "_owner", None) is not None:   # borrowed: the batch destroys it
            self._h = None
            return
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.smc_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != SMC_OK:
            raise SmcError(rc, self._lib.smc_last_error(self._h).decode())

    def eval_likelihood(self, level, theta, want_G=True):
        """Host arrays in and out: returns (G [n, n_obs] or None, Phi [n])."""
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1, self.K)
        n = theta.shape[0]
        G = np.empty((n, self.n_obs)) if want_G else None
        Phi = np.empty(n)
        self._check(self._lib.smc_eval_likelihood(self._h, level, n, _dptr(theta), _dptr(G), _dptr(Phi)))
        return G, Phi

    def eval_likelihood_device(self, level, n, theta_ptr, G_ptr, Phi_ptr, iters_ptr=None, stream=None):
        """Device pointers (ints, e.g. torch tensor data_ptr()); queued on stream, no wait."""
        self._check(self._lib.smc_eval_likelihood_device(self._h, level, n, theta_ptr, G_ptr, Phi_ptr,
                                                         iters_ptr, stream))

    # ---- sampler ------------------------------------------------------------------------
    def step(self):
        info = StageInfo()
        self._check(self._lib.smc_step(self._h, ctypes.byref(info)))
        return info.as_dict()

    def run(self, max_updates=0):
        info = StageInfo()
        self._check(self._lib.smc_run(self._h, int(max_updates), ctypes.byref(info)))
        return info.as_dict()

    def state(self):
        lvl, beta, lz, nu = ctypes.c_int(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        ev = (ctypes.c_longlong * 8)()
        self._check(self._lib.smc_state(self._h, ctypes.byref(lvl), ctypes.byref(beta), ctypes.byref(lz),
                                        ctypes.byref(nu), ev))
        return dict(level=lvl.value, beta=beta.value, log_z=lz.value, n_updates=nu.value, evals=list(ev))

    def surrogate_gate(self, level):
        """The screening gate of one level: (decision 0/1/-1, solve ms, surrogate pass ms)."""
        dec, ts, tp = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        self._check(self._lib.smc_surrogate_gate(self._h, int(level), ctypes.byref(dec), ctypes.byref(ts),
                                                 ctypes.byref(tp)))
        return dec.value, ts.value, tp.value

    def path(self):
        cnt = ctypes.c_int()
        self._check(self._lib.smc_path(self._h, 0, None, ctypes.byref(cnt)))
        arr = (StageInfo * max(cnt.value, 1))()
        self._check(self._lib.smc_path(self._h, cnt.value, arr, ctypes.byref(cnt)))
        return [arr[i].as_dict() for i in range(cnt.value)]

    def posterior_moments(self):
        m, v, lz = np.empty(self.K), np.empty(self.K), ctypes.c_double()
        self._check(self._lib.smc_posterior_moments(self._h, _dptr(m), _dptr(v), ctypes.byref(lz)))
        return m, v, lz.value

    def particles(self):
        th, ph = np.empty((self.J, self.K)), np.empty(self.J)
        self._check(self._lib.smc_get_particles(self._h, _dptr(th), _dptr(ph)))
        return th, ph

    def set_particles(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(self.J, self.K)
        self._check(self._lib.smc_set_particles(self._h, _dptr(theta)))

    def autotune(self, n_tune=1024):
        chosen = (ctypes.c_int * self.n_levels)()
        ms = np.zeros(self.n_levels, dtype=np.float32)
        self._check(self._lib.smc_autotune(self._h, int(n_tune), chosen, ms.ctypes.data))
        return list(chosen), ms.tolist()

    def set_block_size(self, level, T):
        self._check(self._lib.smc_set_block_size(self._h, int(level), int(T)))

    def block_size(self, level):
        """Threads per particle the solves of `level` run with (negative: a compact form)."""
        T = ctypes.c_int()
        self._check(self._lib.smc_block_size(self._h, int(level), ctypes.byref(T)))
        return T.value

    def set_timing(self, enable=True):
        self._check(self._lib.smc_set_timing(self._h, int(bool(enable))))

    def get_timing(self):
        ms = np.zeros(8)
        cnt = (ctypes.c_longlong * 8)()
        self._check(self._lib.smc_get_timing(self._h, _dptr(ms), cnt))
        return ms, list(cnt)

    PHASES = ("surrogate_training", "surrogate_inference", "screening", "reweight_resample", "moves", "gate")

    def get_phase_timing(self):
        """Device milliseconds per phase since the last call (with set_timing(True))."""
        ms = np.zeros(8)
        self._check(self._lib.smc_get_phase_timing(self._h, _dptr(ms)))
        return dict(zip(self.PHASES, ms[:len(self.PHASES)].tolist()))

    def tempering_update(self, level, beta0=0.0, n_mcmc=1):
        info = StageInfo()
        self._check(self._lib.smc_tempering_update(self._h, int(level), float(beta0), int(n_mcmc),
                                                   ctypes.byref(info)))
        return info.as_dict()

    def bridging_update(self, level, beta=1.0, zeta0=0.0, n_mcmc=1):
        info = StageInfo()
        self._check(self._lib.smc_bridging_update(self._h, int(level), float(beta), float(zeta0), int(n_mcmc),
                                                  ctypes.byref(info)))
        return info.as_dict()

    # ---- kernel-level entry points ---------------------------------------------------------
    def next_increment(self, a, dmax):
        a = np.ascontiguousarray(a, dtype=np.float64)
        out = np.empty(3)
        self._check(self._lib.smc_next_increment(self._h, a.size, _dptr(a), float(dmax), _dptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def systematic_resample(self, w, U):
        w = np.ascontiguousarray(w, dtype=np.float64)
        anc = np.empty(w.size, dtype=np.int32)
        self._check(self._lib.smc_systematic_resample(self._h, w.size, _dptr(w), float(U),
                                                      anc.ctypes.data_as(_ip)))
        return anc

    def philox_normals(self, J, K, event, purpose):
        out = np.empty((J, K))
        self._check(self._lib.smc_philox_normals(self._h, J, K, event, purpose, _dptr(out)))
        return out

    def philox_uniforms(self, J, event, purpose):
        out = np.empty(J)
        self._check(self._lib.smc_philox_uniforms(self._h, J, event, purpose, _dptr(out)))
        return out

    # ---- surrogate network -----------------------------------------------------------------
    def surrogate_dims(self):
        d = (ctypes.c_int * 6)()
        self._check(self._lib.smc_surrogate_dims(self._h, d))
        return list(d)

    def _nparams(self):
        d = self.surrogate_dims()
        return sum(d[l + 1] * d[l] + d[l + 1] for l in range(5))

    def unflatten(self, flat):
        d = self.surrogate_dims()
        W, b, off = [], [], 0
        for l in range(5):
            W.append(flat[off:off + d[l + 1] * d[l]].reshape(d[l + 1], d[l]))
            off += d[l + 1] * d[l]
            b.append(flat[off:off + d[l + 1]])
            off += d[l + 1]
        return W, b

    def surrogate_get(self, level):
        p = np.empty(self._nparams(), dtype=np.float32)
        ms = np.empty(2 * self.surrogate_dims()[5], dtype=np.float32)
        self._check(self._lib.smc_surrogate_params(self._h, level, 1, p.ctypes.data, ms.ctypes.data))
        return p, ms

    def surrogate_set(self, level, params, mu_sd):
        p = np.ascontiguousarray(params, dtype=np.float32)
        ms = np.ascontiguousarray(mu_sd, dtype=np.float32)
        self._check(self._lib.smc_surrogate_params(self._h, level, 0, p.ctypes.data, ms.ctypes.data))

    def surrogate_add_pairs(self, level, theta, G):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float64)
        self._check(self._lib.smc_surrogate_add_pairs(self._h, level, theta.shape[0], _dptr(theta), _dptr(G)))

    def surrogate_train(self, level, steps, batch):
        loss = ctypes.c_double()
        self._check(self._lib.smc_surrogate_train(self._h, level, steps, batch, ctypes.byref(loss)))
        return loss.value

    def surrogate_predict(self, level, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        G = np.empty((theta.shape[0], self.n_obs))
        phi = np.empty(theta.shape[0])
        self._check(self._lib.smc_surrogate_predict(self._h, level, theta.shape[0], _dptr(theta), _dptr(G),
                                                    _dptr(phi)))
        return G, phi

    def surrogate_grads(self, level, theta, G):
        theta = np.ascontiguousarray(theta, dtype=np.float64)
        G = np.ascontiguousarray(G, dtype=np.float64)
        g = np.empty(self._nparams(), dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.smc_surrogate_grads(self._h, level, theta.shape[0], _dptr(theta), _dptr(G),
                                                  g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def kl_table(self, level, N):
        psi = np.empty((self.K, 2 * N * N))
        lam = np.empty(self.K)
        self._check(self._lib.smc_kl_table(self._h, level, _dptr(psi), _dptr(lam)))
        return psi, lam
