"""ctypes binding of librihf.so: the C ABI of include/rihf.h with the same names.

Argument marshalling only -- every step of the method runs in the library's CUDA
kernels.  Loading fails loudly when the library is missing; there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librihf.so")

RIHF_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "TIMEOUT",
          -6: "NOT_POSITIVE_DEFINITE", -7: "STATE"}
MAT = dict(S=0, H=1, A=2, LINV=3, T3=4, B=5, J=6, K=7, F=8, D=9, GRAD_PARTS=10, SCHWARZ=11, DPRED=12, FEATURES=13,
           DSAD=14)
PRECISION_FP64, PRECISION_MIXED = 0, 1


class RihfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class rihf_shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("l", ctypes.c_int), ("nprim", ctypes.c_int),
                ("exps", ctypes.POINTER(ctypes.c_double)), ("coefs", ctypes.POINTER(ctypes.c_double))]


class rihf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pure", ctypes.c_int), ("schwarz_tau", ctypes.c_double),
                ("lindep_tau", ctypes.c_double), ("conv_e", ctypes.c_double), ("conv_diis", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("diis_size", ctypes.c_int), ("mixed_digits", ctypes.c_int),
                ("device", ctypes.c_int), ("cuda_graphs", ctypes.c_int), ("confirm_fp64", ctypes.c_int),
                ("aux_chunk", ctypes.c_int)]


EXPORTS = ["rihf_default_options", "rihf_setup", "rihf_update_geometry", "rihf_scf", "rihf_gradient",
           "rihf_query", "rihf_get_matrix", "rihf_screening_stats", "rihf_timings", "rihf_strerror",
           "rihf_last_error", "rihf_destroy", "rihf_eigh", "rihf_stream", "rihf_trace", "rihf_trace_stats",
           "rihf_scf_stats", "rihf_eigh_noalloc", "rihf_tc_dgemm", "rihf_learn_config", "rihf_learn_stats",
           "rihf_mlp_eval", "rihf_learn_params", "rihf_batch_step"]

_lib = None


def load(path: str = LIB_PATH):
    """Load librihf.so (build it with ``paper_2407_19614_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librihf.so not found at %s: build it with python -m paper_2407_19614_gb300.build" % path)
    lib = ctypes.CDLL(path)
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.rihf_default_options.argtypes = [ctypes.POINTER(rihf_options)]
    lib.rihf_default_options.restype = None
    lib.rihf_setup.argtypes = [I, P, P, I, ctypes.POINTER(rihf_shell), I, ctypes.POINTER(rihf_shell), I,
                               ctypes.POINTER(rihf_options), ctypes.POINTER(P)]
    lib.rihf_update_geometry.argtypes = [P, P]
    lib.rihf_scf.argtypes = [P, I, P, P, P, P, P, P]
    lib.rihf_gradient.argtypes = [P, P]
    lib.rihf_query.argtypes = [P, P, P, P, P]
    lib.rihf_get_matrix.argtypes = [P, I, P]
    lib.rihf_screening_stats.argtypes = [P, P, P]
    lib.rihf_timings.argtypes = [P, P]
    lib.rihf_strerror.argtypes = [I]
    lib.rihf_strerror.restype = ctypes.c_char_p
    lib.rihf_last_error.argtypes = []
    lib.rihf_last_error.restype = ctypes.c_char_p
    lib.rihf_scf_stats.argtypes = [P, P, P, P]
    lib.rihf_scf_stats.restype = I
    lib.rihf_stream.argtypes = [P]
    lib.rihf_stream.restype = P
    lib.rihf_trace.argtypes = [P, I]
    lib.rihf_trace.restype = I
    lib.rihf_trace_stats.argtypes = [P, I, P, P, P, P, P]
    lib.rihf_trace_stats.restype = I
    lib.rihf_eigh_noalloc.argtypes = [I, P, P, P, P]
    lib.rihf_eigh_noalloc.restype = I
    lib.rihf_eigh.argtypes = [I, P, P, P, I]
    lib.rihf_eigh.restype = I
    lib.rihf_tc_dgemm.argtypes = [I, I, I, P, P, P, I, I, I]
    lib.rihf_tc_dgemm.restype = I
    lib.rihf_learn_config.argtypes = [P, I, I, I, D, ctypes.c_ulonglong]
    lib.rihf_learn_config.restype = I
    lib.rihf_learn_stats.argtypes = [P, P, P, P, P]
    lib.rihf_learn_stats.restype = I
    lib.rihf_mlp_eval.argtypes = [I, I, P, P, P, ctypes.c_float, I, P, P, P, P, P, I]
    lib.rihf_mlp_eval.restype = I
    lib.rihf_learn_params.argtypes = [P, P]
    lib.rihf_learn_params.restype = I
    lib.rihf_batch_step.argtypes = [I, P, P, I, P, P, P, I]
    lib.rihf_batch_step.restype = I
    lib.rihf_destroy.argtypes = [P]
    lib.rihf_destroy.restype = None
    for name in ("rihf_setup", "rihf_update_geometry", "rihf_scf", "rihf_gradient", "rihf_query",
                 "rihf_get_matrix", "rihf_screening_stats", "rihf_timings"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


def _check(rc, allow=()):
    if rc != RIHF_OK and rc not in allow:
        raise RihfError(rc, load().rihf_last_error().decode())
    return rc


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def default_options(**kw) -> rihf_options:
    o = rihf_options()
    load().rihf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _shells(shells):
    arr = (rihf_shell * len(shells))()
    keep = []
    for i, s in enumerate(shells):
        e = np.ascontiguousarray(s.exps, dtype=np.float64)
        c = np.ascontiguousarray(s.coefs, dtype=np.float64)
        keep += [e, c]
        arr[i].atom, arr[i].l, arr[i].nprim = s.atom, s.l, len(e)
        arr[i].exps = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].coefs = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return arr, keep


def eigh(A, device=0):
    """Eigen-decomposition of a symmetric matrix by the library's eigensolver."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    W = np.zeros(n)
    V = np.zeros((n, n))
    _check(load().rihf_eigh(n, _p(A), _p(W), _p(V), int(device)))
    return W, V


def tc_dgemm(A, B, digits=7, kblock=0, device=0):
    """C = A B^T on the tensor cores from BF16 digit planes (A: M x K, B: N x K)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B need the same number of columns")
    C = np.zeros((M, N))
    _check(load().rihf_tc_dgemm(M, N, K, _p(A), _p(B), _p(C), int(digits), int(kblock), int(device)))
    return C


MLP_F = 12


def mlp_nparams(hidden):
    return hidden * MLP_F + 2 * hidden + 1


def mlp_eval(params, X, t=None, lr=0.0, iters=1, hidden=256, device=0):
    """The learned guess's BF16 network kernels on host arrays: returns dict with
    y (forward) and, with targets t, grad, loss2 and (lr > 0) params after `iters`
    Adam steps with the loss before each step in losses."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    M = X.shape[0]
    y = np.zeros(M, dtype=np.float32)
    out = dict(y=y)
    tt = grad = loss2 = pout = losses = None
    if t is not None:
        tt = np.ascontiguousarray(t, dtype=np.float32)
        grad = np.zeros_like(p)
        loss2 = np.zeros(2, dtype=np.float32)
        out.update(grad=grad, loss2=loss2)
        if lr > 0:
            pout = np.zeros_like(p)
            losses = np.zeros(int(iters), dtype=np.float32)
            out["params"] = pout
            out["losses"] = losses
    _check(load().rihf_mlp_eval(int(hidden), M, _p(p), _p(X), _p(tt), float(lr), int(iters), _p(y), _p(grad),
                                _p(pout), _p(loss2), _p(losses), int(device)))
    return out


def batch_step(contexts, xyz=None, guess=2, nthreads=0):
    """One AIMD step (update geometry, SCF, gradient) for a batch of contexts,
    run concurrently; returns energies, the per-molecule gradients and iterations."""
    n = len(contexts)
    hs = (ctypes.c_void_p * n)(*[c.h.value for c in contexts])
    keep = []
    xp = None
    if xyz is not None:
        arr = (ctypes.c_void_p * n)()
        for i, x in enumerate(xyz):
            if x is not None:
                a = np.ascontiguousarray(x, dtype=np.float64)
                keep.append(a)
                arr[i] = a.ctypes.data
        xp = arr
    E = np.zeros(n)
    it = np.zeros(n, dtype=np.int32)
    sizes = [c.natoms * 3 for c in contexts]
    G = np.zeros(sum(sizes))
    _check(load().rihf_batch_step(n, hs, xp, int(guess), _p(E), _p(G), _p(it), int(nthreads)))
    grads, o = [], 0
    for c, s in zip(contexts, sizes):
        grads.append(G[o:o + s].reshape(c.natoms, 3))
        o += s
    return E, grads, it


def eigh_noalloc(n, A_dev, W_dev, V_dev, stream=0):
    """Allocation-free eigensolver on caller-owned DEVICE buffers (integer
    device addresses, e.g. torch.Tensor.data_ptr()); returns the status code."""
    return load().rihf_eigh_noalloc(int(n), ctypes.c_void_p(A_dev), ctypes.c_void_p(W_dev), ctypes.c_void_p(V_dev),
                                    ctypes.c_void_p(stream) if stream else None)


class Context:
    """Owns one rihf_ctx (one molecule on one GPU)."""

    def __init__(self, mol, options: rihf_options | None = None, **kw):
        lib = load()
        self.lib = lib
        opt = options or default_options(**kw)
        Z = np.ascontiguousarray(mol.Z, dtype=np.int32)
        xyz = np.ascontiguousarray(mol.xyz, dtype=np.float64)
        prim, k1 = _shells(mol.primary)
        aux, k2 = _shells(mol.aux)
        h = ctypes.c_void_p()
        _check(lib.rihf_setup(len(Z), _p(Z), _p(xyz), len(mol.primary), prim, len(mol.aux), aux,
                              int(Z.sum()), ctypes.byref(opt), ctypes.byref(h)))
        self.h = h
        N, NA, no, na = (ctypes.c_int() for _ in range(4))
        lib.rihf_query(h, ctypes.byref(N), ctypes.byref(NA), ctypes.byref(no), ctypes.byref(na))
        self.N, self.Naux, self.nocc, self.natoms = N.value, NA.value, no.value, na.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.rihf_destroy(self.h)
            self.h = None

    __del__ = close

    def learn_config(self, hidden=256, train_steps=200, adam_iters=4, lr=1e-3, seed=0):
        _check(self.lib.rihf_learn_config(self.h, int(hidden), int(train_steps), int(adam_iters), float(lr),
                                          int(seed)))
        self._hidden = int(hidden)

    def learn_stats(self):
        n, g = ctypes.c_int(), ctypes.c_int()
        r, sc = ctypes.c_double(), ctypes.c_double()
        self.lib.rihf_learn_stats(self.h, ctypes.byref(n), ctypes.byref(r), ctypes.byref(g), ctypes.byref(sc))
        return dict(trained_steps=n.value, last_ratio=r.value, last_guess=g.value, scale=sc.value)

    def learn_params(self, hidden=None):
        n = mlp_nparams(hidden or self._hidden)
        out = np.zeros(n, dtype=np.float32)
        _check(self.lib.rihf_learn_params(self.h, _p(out)))
        return out

    def update_geometry(self, xyz):
        x = np.ascontiguousarray(xyz, dtype=np.float64)
        _check(self.lib.rihf_update_geometry(self.h, _p(x)))

    def scf(self, guess=0, C_guess=None, outputs=True, allow_unconverged=False):
        N = self.N
        e = np.zeros(1)
        it = np.zeros(1, dtype=np.int32)
        D = np.zeros((N, N)) if outputs else None
        C = np.zeros((N, N)) if outputs else None
        eps = np.zeros(N) if outputs else None
        Cg = np.ascontiguousarray(C_guess, dtype=np.float64) if C_guess is not None else None
        rc = self.lib.rihf_scf(self.h, int(guess), _p(Cg), _p(e), _p(D), _p(C), _p(eps), _p(it))
        _check(rc, allow=(-4,) if allow_unconverged else ())
        return dict(energy=float(e[0]), D=D, C=C, eps=eps, iterations=int(it[0]), converged=(rc == 0))

    def gradient(self):
        g = np.zeros((self.natoms, 3))
        _check(self.lib.rihf_gradient(self.h, _p(g)))
        return g

    def matrix(self, name):
        N, NA = self.N, self.Naux
        shapes = dict(S=(N, N), H=(N, N), J=(N, N), K=(N, N), F=(N, N), D=(N, N), A=(NA, NA), LINV=(NA, NA),
                      T3=(NA, N, N), B=(NA, N, N), GRAD_PARTS=(5, self.natoms, 3),
                      SCHWARZ=(self.screening_stats()[1],), DPRED=(N, N), FEATURES=(N * (N + 1) // 2, MLP_F),
                      DSAD=(N, N))
        out = np.zeros(shapes[name])
        _check(self.lib.rihf_get_matrix(self.h, MAT[name], _p(out)))
        return out

    def screening_stats(self):
        k, t = ctypes.c_int(), ctypes.c_int()
        _check(self.lib.rihf_screening_stats(self.h, ctypes.byref(k), ctypes.byref(t)))
        return k.value, t.value

    def scf_stats(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.lib.rihf_scf_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(tc_builds=a.value, fp64_builds=b.value, confirm_builds=c.value)

    def stream(self) -> int:
        """cudaStream_t of the context (as an integer handle)."""
        return int(self.lib.rihf_stream(self.h) or 0)

    def trace(self, enable: bool):
        _check(self.lib.rihf_trace(self.h, int(bool(enable))))

    def trace_stats(self, max_kernels=64):
        names = ctypes.create_string_buffer(48 * max_kernels)
        la, ms, wk = np.zeros(max_kernels), np.zeros(max_kernels), np.zeros(max_kernels)
        kind = np.zeros(max_kernels, dtype=np.int32)
        n = self.lib.rihf_trace_stats(self.h, max_kernels, names, _p(la), _p(ms), _p(wk), _p(kind))
        out = []
        for i in range(n):
            nm = names.raw[48 * i:48 * (i + 1)].split(b"\0")[0].decode()
            out.append(dict(name=nm, launches=int(la[i]), ms=float(ms[i]), work=float(wk[i]),
                            kind=["fp64_flops", "hbm_bytes", "fp32_flops", "bf16_tensor_flops"][int(kind[i])]))
        return out

    def timings(self):
        t = np.zeros(5)
        _check(self.lib.rihf_timings(self.h, _p(t)))
        return dict(integrals_ms=t[0], fock_ms=t[1], diag_ms=t[2], gradient_ms=t[3], launches=int(t[4]))
