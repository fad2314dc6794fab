"""Thin Python binding of the libdopinf C ABI (include/dopinf.h).

Argument marshalling only: every step of the hot path runs in the CUDA library.  Device
memory, workspaces and streams come from PyTorch; tensors are passed by data pointer.  The
functions keep the C names.  Importing this module loads libdopinf.so and raises if it is
missing - there is no fallback.

Layout convention: the snapshot matrix is column-major, i.e. a torch tensor of shape (n, k)
with strides (1, ldq); ``snapshot_matrix(n, k)`` allocates one, and ``QT.t()`` of a row-major
(k, n) tensor is one.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdopinf.so")

OK, E_ARG, E_CUDA, E_NONFINITE, E_RANK, E_NO_STABLE, E_TIMEOUT, E_UNSUPPORTED = 0, -1, -2, -4, -6, -7, -8, -9
FLAG_NONFINITE, FLAG_ZERO_SCALE, FLAG_TIMEOUT, FLAG_RANK, FLAG_NO_STABLE = 1, 2, 4, 8, 16
F64, F32 = 0, 1
CENTER, SCALE, SCALE_STD = 1, 2, 4
GRAM_FP64, GRAM_BF16X4, GRAM_OZAKI_FP64 = 0, 1, 2
DISCRETE, CONTINUOUS_RK4 = 0, 1
ROLLOUT_FP64, ROLLOUT_DW = 1, 2
TEST_GRID_BARRIER, TEST_TENSOR_GRAM = 1, 2
SOLVE_CHOLESKY, SOLVE_QR = 0, 1

_c_i64 = ctypes.c_int64
_c_p = ctypes.c_void_p
_c_sz = ctypes.c_size_t


class DopinfError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        detail = lib.dopinf_last_error().decode() if status == E_CUDA else ""
        super().__init__("%s failed: %d (%s)%s" % (fn, status, status_string(status),
                                                    " - " + detail if detail else ""))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdopinf.so is not built (run __graft_entry__.build()); "
                          "the dOpInf hot path has no non-CUDA fallback")
    lib = ctypes.CDLL(LIB_PATH)
    sig = {
        "dopinf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "dopinf_last_error": (ctypes.c_char_p, []),
        "dopinf_transform_workspace": (_c_sz, [_c_i64, ctypes.c_int]),
        "dopinf_transform": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, _c_i64, ctypes.c_int,
                                            ctypes.POINTER(_c_i64), ctypes.c_uint, _c_p, _c_p, _c_p,
                                            _c_p, _c_sz, _c_p]),
        "dopinf_gram_workspace": (_c_sz, [_c_i64, _c_i64, ctypes.c_int, ctypes.c_int]),
        "dopinf_gram": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, _c_i64, ctypes.c_int,
                                       ctypes.c_int, _c_p, _c_i64, _c_p, _c_sz, _c_p]),
        "dopinf_gram_async": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, _c_i64, ctypes.c_int,
                                             ctypes.c_int, _c_p, _c_i64, _c_p, _c_p, _c_sz, _c_p]),
        "dopinf_reduce_async": (ctypes.c_int, [_c_p, _c_i64, _c_i64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p]),
        "dopinf_learn_async": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_int),
                                              ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_double, _c_i64, ctypes.c_double, _c_p, _c_p, _c_p, _c_p,
                                              _c_p, _c_p, _c_p, _c_p, _c_sz, _c_p]),
        "dopinf_reduce_workspace": (_c_sz, [_c_i64, ctypes.c_int]),
        "dopinf_reduce": (ctypes.c_int, [_c_p, _c_i64, _c_i64, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), _c_p, _c_p, _c_p, _c_p,
                                         _c_sz, _c_p]),
        "dopinf_learn_workspace": (_c_sz, [ctypes.c_int, _c_i64, ctypes.POINTER(ctypes.c_int),
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "dopinf_learn": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, ctypes.POINTER(ctypes.c_int),
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _c_i64, ctypes.c_double, _c_p, _c_p, _c_p, _c_p,
                                        ctypes.POINTER(ctypes.c_int), _c_p, ctypes.POINTER(ctypes.c_double), _c_p,
                                        _c_sz, _c_p]),
        "dopinf_learn_operator_offset": (_c_sz, [_c_i64, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int]),
        "dopinf_lift_workspace": (_c_sz, [_c_i64, ctypes.c_int]),
        "dopinf_lift": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, _c_i64, _c_p, _c_i64, ctypes.c_int, _c_p,
                                       _c_i64, _c_i64, _c_p, _c_i64, _c_p, _c_p, ctypes.c_int, ctypes.POINTER(_c_i64),
                                       _c_p, _c_i64, _c_p, _c_sz, _c_p]),
        "dopinf_gram_host_workspace": (_c_sz, [_c_i64, _c_i64, ctypes.c_int, ctypes.c_int]),
        "dopinf_gram_host": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_i64, _c_i64, ctypes.c_int, ctypes.c_int, _c_p,
                                            _c_i64, _c_i64, _c_p, _c_sz, _c_p]),
        "dopinf_mlp_feature_stats": (ctypes.c_int, [_c_p, ctypes.c_int, _c_p, _c_p, _c_p]),
        "dopinf_mlp_standardize": (ctypes.c_int, [_c_p, ctypes.c_int, _c_p, _c_p, _c_p, _c_p]),
        "dopinf_mlp_rank": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, _c_p, _c_p,
                                           _c_p]),
        "dopinf_tune_learn_solver": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_tune_gram_chunk": (_c_i64, [_c_i64]),
        "dopinf_test_expire_waits": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_tune_rollout_rows_large": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_tune_rollout_rows": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_tune_rollout_arith": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_tune_reduce_coop": (ctypes.c_int, [ctypes.c_int]),
        "dopinf_rollout": (ctypes.c_int, [_c_p, ctypes.c_int, _c_i64, _c_p, _c_i64, ctypes.c_int,
                                          ctypes.c_double, _c_p, _c_p, _c_p]),
        "dopinf_proposal_features": (ctypes.c_int, [_c_p, ctypes.c_int, ctypes.c_double, _c_p, ctypes.c_int,
                                                    _c_i64, _c_i64, _c_p, _c_p]),
        "dopinf_mlp_param_count": (_c_sz, [ctypes.c_int]),
        "dopinf_mlp_workspace": (_c_sz, [ctypes.c_int, ctypes.c_int]),
        "dopinf_mlp_forward": (ctypes.c_int, [_c_p, ctypes.c_int, _c_p, ctypes.c_int, _c_p, _c_p, _c_sz, _c_p]),
        "dopinf_mlp_train_step": (ctypes.c_int, [_c_p, _c_p, _c_p, ctypes.c_int, ctypes.c_float,
                                                 ctypes.POINTER(ctypes.c_int), _c_p, _c_p, ctypes.c_int, _c_p, _c_p,
                                                 _c_p, _c_sz, _c_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def status_string(status):
    return lib.dopinf_status_string(int(status)).decode()


def _check(fn, status, allowed=(OK,)):
    if status not in allowed:
        raise DopinfError(fn, status)
    return status


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Workspace:
    """Reusable device workspace (256-byte aligned) grown on demand."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes):
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.buf.data_ptr()) % 256
        return self.buf[off:off + nbytes]


_default_ws = {}


def _ws(nbytes, ws, device):
    if ws is None:
        ws = _default_ws.setdefault(str(device), Workspace(device))
    buf = ws.get(nbytes)
    return buf, nbytes


def snapshot_matrix(n, k, dtype=torch.float64, device="cuda"):
    """Column-major (n, k) tensor: snapshot t is contiguous."""
    return torch.empty(k, n, dtype=dtype, device=device).t()


def _colmajor(Q):
    n, k = Q.shape
    if Q.stride(0) != 1 or (k > 1 and Q.stride(1) < max(n, 1)):
        raise ValueError("expected a column-major (n, k) tensor with strides (1, ldq >= n)")
    return n, k, Q.stride(1) if k > 1 else max(n, 1)


def _dtype_code(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError("snapshot data must be float64 or float32")


def dopinf_transform(Q, var_row_offsets, flags=CENTER | SCALE, dev_flags=None, ws=None, stream=None):
    """Step II in place on Q; returns (row_mean, var_scale, dev_flags)."""
    n, k, ldq = _colmajor(Q)
    offs = (_c_i64 * len(var_row_offsets))(*[int(v) for v in var_row_offsets])
    n_vars = len(var_row_offsets) - 1
    mean = torch.empty(n, dtype=torch.float64, device=Q.device)
    scale = torch.empty(n_vars, dtype=torch.float64, device=Q.device)
    if dev_flags is None:
        dev_flags = torch.zeros(1, dtype=torch.int32, device=Q.device)
    nb = lib.dopinf_transform_workspace(n, n_vars)
    buf, nb = _ws(nb, ws, Q.device)
    _check("dopinf_transform", lib.dopinf_transform(_ptr(Q), _dtype_code(Q), n, k, ldq, n_vars, offs, flags,
                                                    _ptr(mean), _ptr(scale), _ptr(dev_flags), _ptr(buf), nb,
                                                    _stream(stream)))
    return mean, scale, dev_flags


def dopinf_gram(Q, mode=GRAM_FP64, D=None, accumulate=False, ws=None, stream=None):
    """Step III Gram D = Q^T Q (k x k FP64); with accumulate, D += Q^T Q."""
    n, k, ldq = _colmajor(Q)
    if D is None:
        D = torch.zeros(k, k, dtype=torch.float64, device=Q.device)
    nb = lib.dopinf_gram_workspace(n, k, _dtype_code(Q), mode)
    buf, nb = _ws(nb, ws, Q.device)
    # D is symmetric, so its row-major storage is its column-major storage
    _check("dopinf_gram", lib.dopinf_gram(_ptr(Q), _dtype_code(Q), n, k, ldq, mode, int(accumulate), _ptr(D),
                                          D.stride(0), _ptr(buf), nb, _stream(stream)))
    return D


def dopinf_gram_host(Q_host, chunk_rows, mode=GRAM_FP64, D=None, accumulate=False, ws=None, stream=None,
                     device="cuda"):
    """Out-of-core Gram of a snapshot matrix in host memory: Q_host is a CPU (n, k) column-major
    tensor (pinned for overlapped copies), streamed in row blocks of chunk_rows; D (k x k FP64)
    on the device."""
    if Q_host.is_cuda:
        raise ValueError("Q_host must be in host memory")
    n, k, ldq = _colmajor(Q_host)
    if D is None:
        D = torch.zeros(k, k, dtype=torch.float64, device=device)
    nb = lib.dopinf_gram_host_workspace(min(int(chunk_rows), n), k, _dtype_code(Q_host), mode)
    buf, nb = _ws(nb, ws, D.device)
    _check("dopinf_gram_host", lib.dopinf_gram_host(_ptr(Q_host), _dtype_code(Q_host), n, k, ldq, mode,
                                                    int(accumulate), _ptr(D), D.stride(0), int(chunk_rows), _ptr(buf),
                                                    nb, _stream(stream)))
    return D


def dopinf_gram_async(Q, D, flags, mode=GRAM_FP64, accumulate=False, ws=None, stream=None):
    """dopinf_gram without synchronisation (capturable): a kernel timeout ORs FLAG_TIMEOUT into
    the device word `flags` (int32 tensor of one element)."""
    n, k, ldq = _colmajor(Q)
    nb = lib.dopinf_gram_workspace(n, k, _dtype_code(Q), mode)
    buf, nb = _ws(nb, ws, Q.device)
    _check("dopinf_gram_async", lib.dopinf_gram_async(_ptr(Q), _dtype_code(Q), n, k, ldq, mode, int(accumulate),
                                                      _ptr(D), D.stride(0), _ptr(flags), _ptr(buf), nb,
                                                      _stream(stream)))
    return D


def dopinf_tune_gram_chunk(rows=0):
    """Sets (rows > 0) or queries the FP32 accumulation chunk of the split Gram; returns the previous value."""
    return int(lib.dopinf_tune_gram_chunk(int(rows)))


def dopinf_tune_learn_solver(solver=-1):
    """Sets (SOLVE_CHOLESKY, SOLVE_QR) or queries the solver of the regularised problems of
    dopinf_learn; returns the previous value."""
    return int(lib.dopinf_tune_learn_solver(int(solver)))


def dopinf_test_expire_waits(which=-1):
    """Test of the error paths: withholds the signal of the named bounded waits (TEST_GRID_BARRIER,
    TEST_TENSOR_GRAM) so that they expire; 0 restores; returns the previous value."""
    return int(lib.dopinf_test_expire_waits(int(which)))


def dopinf_tune_rollout_rows_large(rows=0):
    """Sets (3 to 8) or queries the operator rows per CTA of the rollouts of 32 < r <= 92 (the
    cluster of one candidate has ceil(r / rows) CTAs, at most 16); returns the previous value."""
    return int(lib.dopinf_tune_rollout_rows_large(int(rows)))


def dopinf_tune_rollout_arith(arith=0):
    """Sets (ROLLOUT_FP64, ROLLOUT_DW) or queries the arithmetic of the learn rollouts; returns
    the previous value."""
    return int(lib.dopinf_tune_rollout_arith(int(arith)))


def dopinf_tune_rollout_rows(rows=0):
    """Sets (1, 2, 4, 8) or queries the operator rows per CTA of the rollouts of r <= 32 (the
    cluster of one candidate has ceil(r / rows) CTAs, at most 16); returns the previous value."""
    return int(lib.dopinf_tune_rollout_rows(int(rows)))


def dopinf_tune_reduce_coop(on=-1):
    """Sets (1: one cooperative launch, 0: three launches per column) or queries the
    tridiagonalisation of dopinf_reduce; returns the previous value."""
    return int(lib.dopinf_tune_reduce_coop(int(on)))


def dopinf_reduce(D, r_cap, energy_target=0.9996, r_fixed=0, ws=None, stream=None):
    """Step III eigensolve/projection.  Returns dict(r, trace, eigvals, Tr (k x r_cap), Qhat (r_cap x k)).

    Qhat is returned as an (r_cap, k) tensor whose column t is the reduced snapshot t.
    """
    k = D.shape[0]
    dev = D.device
    eig = torch.empty(r_cap, dtype=torch.float64, device=dev)
    Tr = torch.empty(r_cap, k, dtype=torch.float64, device=dev).t()       # k x r_cap column-major
    Qhat = torch.empty(k, r_cap, dtype=torch.float64, device=dev).t()     # r_cap x k column-major
    r = ctypes.c_int(0)
    tr = ctypes.c_double(0.0)
    nb = lib.dopinf_reduce_workspace(k, r_cap)
    buf, nb = _ws(nb, ws, dev)
    st = lib.dopinf_reduce(_ptr(D), k, D.stride(0), float(energy_target), int(r_fixed), int(r_cap),
                           ctypes.byref(r), ctypes.byref(tr), _ptr(eig), _ptr(Tr), _ptr(Qhat), _ptr(buf), nb,
                           _stream(stream))
    _check("dopinf_reduce", st)
    return dict(r=r.value, trace=tr.value, eigvals=eig, Tr=Tr, Qhat=Qhat, status=st)


def dopinf_reduce_async(D, r_cap, out, energy_target=0.9996, r_fixed=0, ws=None, stream=None):
    """dopinf_reduce without synchronisation (capturable).  `out` holds preallocated device
    tensors: eigvals (r_cap), Tr (k x r_cap column-major), Qhat (r_cap x k column-major),
    r (int32, 1), trace (float64, 1), flags (int32, 1)."""
    k = D.shape[0]
    nb = lib.dopinf_reduce_workspace(k, r_cap)
    buf, nb = _ws(nb, ws, D.device)
    _check("dopinf_reduce_async",
           lib.dopinf_reduce_async(_ptr(D), k, D.stride(0), float(energy_target), int(r_fixed), int(r_cap),
                                   _ptr(out["r"]), _ptr(out["trace"]), _ptr(out["eigvals"]), _ptr(out["Tr"]),
                                   _ptr(out["Qhat"]), _ptr(out["flags"]), _ptr(buf), nb, _stream(stream)))
    return out


def dopinf_learn_async(Qhat, r_list, beta1, beta2, n_steps, out, mode=DISCRETE, dt=1.0, max_growth=1.2, ws=None,
                       stream=None):
    """dopinf_learn without synchronisation (capturable).  `out` holds preallocated device
    tensors: train_err, growth (float64, n_cand), status (int32, n_cand), steps (int64,
    n_cand), best (int32, 1), O_best (r_max x d_max column-major), flags (int32, 1)."""
    r_max, k = Qhat.shape
    rl = (ctypes.c_int * len(r_list))(*[int(r) for r in r_list])
    b1 = (ctypes.c_double * len(beta1))(*[float(b) for b in beta1])
    b2 = (ctypes.c_double * len(beta2))(*[float(b) for b in beta2])
    nb = lib.dopinf_learn_workspace(r_max, k, rl, len(r_list), len(beta1), len(beta2))
    buf, nb = _ws(nb, ws, Qhat.device)
    O = out["O_best"]
    _check("dopinf_learn_async",
           lib.dopinf_learn_async(_ptr(Qhat), r_max, k, Qhat.stride(1), rl, len(r_list), b1, len(beta1), b2,
                                  len(beta2), int(mode), float(dt), int(n_steps), float(max_growth),
                                  _ptr(out["train_err"]), _ptr(out["growth"]), _ptr(out["status"]),
                                  _ptr(out["steps"]), _ptr(out["best"]), _ptr(O), _ptr(out["flags"]), _ptr(buf),
                                  nb, _stream(stream)))
    return out


def dopinf_learn(Qhat, r_list, beta1, beta2, n_steps, mode=DISCRETE, dt=1.0, max_growth=1.2, ws=None,
                 stream=None, allow_no_stable=True, operators=False):
    """Step IV grid search.  Qhat: (r_max, k) column-major.  Returns a dict of results; with
    operators=True also "operators": every candidate's (r, d) operator [A | H | c] copied out of
    the workspace (None where its Cholesky factorisation failed)."""
    r_max, k = Qhat.shape
    if Qhat.stride(0) != 1:
        raise ValueError("Qhat must be column-major (r_max, k)")
    ldqh = Qhat.stride(1)
    dev = Qhat.device
    rl = (ctypes.c_int * len(r_list))(*[int(r) for r in r_list])
    b1 = (ctypes.c_double * len(beta1))(*[float(b) for b in beta1])
    b2 = (ctypes.c_double * len(beta2))(*[float(b) for b in beta2])
    n_cand = len(r_list) * len(beta1) * len(beta2)
    err = torch.empty(n_cand, dtype=torch.float64, device=dev)
    gro = torch.empty(n_cand, dtype=torch.float64, device=dev)
    cst = torch.empty(n_cand, dtype=torch.int32, device=dev)
    steps = torch.zeros(n_cand, dtype=torch.int64, device=dev)
    stage = (ctypes.c_double * 3)()
    d_max = max(r + r * (r + 1) // 2 + 1 for r in r_list)
    O_best = torch.zeros(d_max, r_max, dtype=torch.float64, device=dev).t()  # r_max x d_max column-major
    best = ctypes.c_int(-1)
    nb = lib.dopinf_learn_workspace(r_max, k, rl, len(r_list), len(beta1), len(beta2))
    buf, nb = _ws(nb, ws, dev)
    st = lib.dopinf_learn(_ptr(Qhat), r_max, k, ldqh, rl, len(r_list), b1, len(beta1), b2, len(beta2), int(mode),
                          float(dt), int(n_steps), float(max_growth), _ptr(err), _ptr(gro), _ptr(cst),
                          _ptr(steps), ctypes.byref(best), _ptr(O_best), stage, _ptr(buf), nb, _stream(stream))
    _check("dopinf_learn", st, (OK, E_NO_STABLE) if allow_no_stable else (OK,))
    out = dict(train_err=err, growth=gro, status=cst, steps=steps, best=best.value, O_best=O_best, code=st,
               stage_ms=dict(normal_equations=stage[0], solves=stage[1], rollouts=stage[2]))
    if operators:
        stat = cst.cpu().tolist()
        nb12 = len(beta1) * len(beta2)
        ops = []
        for c in range(n_cand):
            r = int(r_list[c // nb12])
            d = r + r * (r + 1) // 2 + 1
            off = lib.dopinf_learn_operator_offset(k, rl, len(r_list), len(beta1), len(beta2), c)
            if stat[c] == 1:
                ops.append(None)
                continue
            flat = buf[off:off + 8 * r * d].view(torch.float64)
            ops.append(flat.view(d, r).t().clone())      # column-major r x d
        out["operators"] = ops
    if best.value >= 0:
        nb12 = len(beta1) * len(beta2)
        r = int(r_list[best.value // nb12])
        out.update(r=r, beta1=float(beta1[(best.value % nb12) // len(beta2)]),
                   beta2=float(beta2[best.value % len(beta2)]),
                   O=O_best[:r, :r + r * (r + 1) // 2 + 1])
    return out


def dopinf_rollout(O, q0, n_steps, mode=DISCRETE, dt=1.0, stream=None):
    """Rollout of one ROM.  O: (r, d) column-major view; returns (Qtilde (n_steps x r), finite)."""
    r, d = O.shape
    if O.stride(0) != 1:
        raise ValueError("O must be column-major (r, d)")
    Qt = torch.full((n_steps, r), float("nan"), dtype=torch.float64, device=O.device)
    fin = torch.zeros(1, dtype=torch.int32, device=O.device)
    q0 = q0.contiguous()
    _check("dopinf_rollout", lib.dopinf_rollout(_ptr(O), r, O.stride(1) if d > 1 else r, _ptr(q0), int(n_steps),
                                                int(mode), float(dt), _ptr(Qt), _ptr(fin), _stream(stream)))
    return Qt, fin


def dopinf_lift(Q, Tr, Qtilde, rows=None, n_rows=None, row_mean=None, var_scale=None, var_row_offsets=None,
                ws=None, stream=None):
    """Step V: the reduced solution lifted at chosen rows.  Q: (n, k) column-major transformed
    snapshots; Tr: (k, r) column-major; Qtilde: (r, n_t) column-major (a (n_t, r) row-major
    trajectory .t() is one); rows: int64 device tensor of row indices, or None for the first
    n_rows rows (default all).  Returns X (n_rows, n_t) column-major."""
    n, k, ldq = _colmajor(Q)
    if Tr.stride(0) != 1 or Qtilde.stride(0) != 1:
        raise ValueError("Tr and Qtilde must be column-major")
    r = Tr.shape[1]
    n_t = Qtilde.shape[1]
    if Qtilde.shape[0] != r:
        raise ValueError("Qtilde must have r rows")
    if rows is not None:
        rows = rows.to(device=Q.device, dtype=torch.int64).contiguous()
        nr = rows.numel()
    else:
        nr = n if n_rows is None else int(n_rows)
    X = torch.empty(n_t, nr, dtype=torch.float64, device=Q.device).t()
    offs = None
    n_vars = 0
    if var_row_offsets is not None:
        n_vars = len(var_row_offsets) - 1
        offs = (_c_i64 * len(var_row_offsets))(*[int(v) for v in var_row_offsets])
    nb = lib.dopinf_lift_workspace(nr, r)
    buf, nb = _ws(nb, ws, Q.device)
    _check("dopinf_lift", lib.dopinf_lift(_ptr(Q), _dtype_code(Q), n, k, ldq, _ptr(Tr), Tr.stride(1) if r > 1 else k,
                                          r, _ptr(Qtilde), Qtilde.stride(1) if n_t > 1 else r, n_t, _ptr(rows), nr,
                                          _ptr(row_mean), _ptr(var_scale), n_vars, offs, _ptr(X), X.stride(1)
                                          if n_t > 1 else nr, _ptr(buf), nb, _stream(stream)))
    return X


# ------------------------------------------------------------------------------ proposal network
def dopinf_proposal_features(eigvals, trace, Qhat, stream=None):
    """64 FP32 features (device tensor) of a reduced system."""
    r_max, k = Qhat.shape
    f = torch.empty(64, dtype=torch.float32, device=Qhat.device)
    eig = eigvals.contiguous()
    _check("dopinf_proposal_features", lib.dopinf_proposal_features(_ptr(eig), eig.numel(), float(trace), _ptr(Qhat),
                                                                    r_max, k, Qhat.stride(1), _ptr(f), _stream(stream)))
    return f


def dopinf_mlp_param_count(n_out):
    return int(lib.dopinf_mlp_param_count(int(n_out)))


def dopinf_mlp_forward(params, n_out, X, ws=None, stream=None):
    B = X.shape[0]
    logits = torch.empty(B, n_out, dtype=torch.float32, device=X.device)
    nb = lib.dopinf_mlp_workspace(B, n_out)
    buf, nb = _ws(nb, ws, X.device)
    _check("dopinf_mlp_forward", lib.dopinf_mlp_forward(_ptr(params), n_out, _ptr(X.contiguous()), B, _ptr(logits),
                                                        _ptr(buf), nb, _stream(stream)))
    return logits


def dopinf_mlp_train_step(params, m, v, step, lr, head_sizes, X, labels, want_grad=False, ws=None, stream=None):
    """One forward/backward/Adam step in place on params, m, v; returns (loss tensor, grad or None)."""
    B = X.shape[0]
    n_out = sum(head_sizes)
    hs = (ctypes.c_int * 3)(*[int(h) for h in head_sizes])
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    grad = torch.empty(dopinf_mlp_param_count(n_out), dtype=torch.float32, device=X.device) if want_grad else None
    nb = lib.dopinf_mlp_workspace(B, n_out)
    buf, nb = _ws(nb, ws, X.device)
    _check("dopinf_mlp_train_step", lib.dopinf_mlp_train_step(_ptr(params), _ptr(m), _ptr(v), int(step), float(lr), hs,
                                                              _ptr(X.contiguous()), _ptr(labels.contiguous()), B,
                                                              _ptr(loss), _ptr(grad), _ptr(buf), nb, _stream(stream)))
    return loss, grad


def dopinf_mlp_feature_stats(X, stream=None):
    """Per-feature mean and sample standard deviation (floored at 1e-6) of X (batch x 64 FP32):
    two FP64 device tensors of 64."""
    X = X.contiguous()
    mu = torch.empty(64, dtype=torch.float64, device=X.device)
    sd = torch.empty(64, dtype=torch.float64, device=X.device)
    _check("dopinf_mlp_feature_stats", lib.dopinf_mlp_feature_stats(_ptr(X), X.shape[0], _ptr(mu), _ptr(sd),
                                                                    _stream(stream)))
    return mu, sd


def dopinf_mlp_standardize(X, mu, sd, stream=None):
    """(X - mu) / sd per feature (FP64 arithmetic, FP32 result)."""
    X = X.contiguous()
    Xs = torch.empty_like(X)
    _check("dopinf_mlp_standardize", lib.dopinf_mlp_standardize(_ptr(X), X.shape[0], _ptr(mu.contiguous()),
                                                                _ptr(sd.contiguous()), _ptr(Xs), _stream(stream)))
    return Xs


def dopinf_mlp_rank(logits, head_sizes, top, stream=None):
    """The `top` grid candidates of each row by joint log-probability: (ranked (batch, top, 3)
    int32, score (batch, top) float64), device tensors."""
    logits = logits.contiguous()
    B = logits.shape[0]
    hs = (ctypes.c_int * 3)(*[int(h) for h in head_sizes])
    ranked = torch.empty(B, top, 3, dtype=torch.int32, device=logits.device)
    score = torch.empty(B, top, dtype=torch.float64, device=logits.device)
    _check("dopinf_mlp_rank", lib.dopinf_mlp_rank(_ptr(logits), B, hs, int(top), _ptr(ranked), _ptr(score),
                                                  _stream(stream)))
    return ranked, score
