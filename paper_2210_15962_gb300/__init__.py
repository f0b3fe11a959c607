"""GB300 (sm_103a) parallel self-avoiding walks for skew-symmetric LABS.

Thin Python binding of the C ABI in ``include/labs.h`` (same names).  This
module only marshals arguments: every step of the solver runs in the CUDA
kernels of ``liblabs_gb300.so``.  There is no CPU fallback; if the library
has not been built (``python -m paper_2210_15962_gb300.build``) or no CUDA
device is usable, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB_PATH

LABS_OK = 0
LABS_PENDING = 1
LABS_EINVAL = -1
LABS_ENOMEM = -2
LABS_ECUDA = -3
LABS_ETIMEOUT = -4
LABS_EOVERFLOW = -5
LABS_ENOTFOUND = -6
LABS_ECHECK = -7
LABS_ESHUTDOWN = -8
WALK_MODE_AUTO = 0
WALK_MODE_LANE = 1
WALK_MODE_WARP = 2
WALK_MODE_CTA = 3  # batches only: one walk per CTA of 128 threads
LABS_L_MIN = 5
LABS_L_MAX = 511
KERNEL_AUTO = 0
KERNEL_FULL_SCAN = 1
KERNEL_INCREMENTAL = 2
KERNEL_WARP = 3
KERNEL_CTA = 4


class LabsError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, status_str(status) if _lib else "?", status))


class labs_opts(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p),
        ("device_buffers", ctypes.c_int32),
        ("recheck_every", ctypes.c_int32),
        ("target_E", ctypes.c_int64),
        ("max_rounds", ctypes.c_int32),
        ("kernel", ctypes.c_int32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("evals_per_seed", ctypes.c_void_p),
        ("rounds_per_seed", ctypes.c_void_p),
    ]


class labs_stats(ctypes.Structure):
    _fields_ = [
        ("evals", ctypes.c_uint64),
        ("rounds", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("walk_launches", ctypes.c_int32),
        ("reserved0", ctypes.c_int32),
        ("walk_kernel_ms", ctypes.c_double),
        ("device_ms", ctypes.c_double),
        ("plane_steps", ctypes.c_uint64),
    ]

    def as_dict(self) -> dict:
        return {f[0]: getattr(self, f[0]) for f in self._fields_ if not f[0].startswith("reserved")}


class labs_problem(ctypes.Structure):
    _fields_ = [
        ("L", ctypes.c_int32),
        ("walks", ctypes.c_int32),
        ("walk_len", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("step_budget", ctypes.c_uint64),
        ("target_E", ctypes.c_int64),
    ]


class labs_batch_opts(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p),
        ("use_graph", ctypes.c_int32),
        ("autotune", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("table_factor_x10", ctypes.c_int32),
        ("rounds_per_launch", ctypes.c_int32),
        ("walk_mode", ctypes.c_int32),
    ]


class labs_serve_cfg(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p),
        ("mem_bytes", ctypes.c_size_t),
        ("max_active", ctypes.c_int32),
        ("max_L", ctypes.c_int32),
        ("max_walks", ctypes.c_int32),
        ("max_walk_len", ctypes.c_int32),
        ("rounds_per_launch", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("walk_mode", ctypes.c_int32),
    ]


class labs_result(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("best_E", ctypes.c_int64),
        ("F", ctypes.c_double),
        ("evals", ctypes.c_uint64),
        ("rounds", ctypes.c_int32),
        ("reached_target", ctypes.c_int32),
        ("t_submit_ns", ctypes.c_uint64),
        ("t_admit_ns", ctypes.c_uint64),
        ("t_done_ns", ctypes.c_uint64),
        ("p_optimal", ctypes.c_double),
        ("plane_steps", ctypes.c_uint64),
    ]


class labs_serve_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_uint64),
        ("completed", ctypes.c_uint64),
        ("pending", ctypes.c_uint64),
        ("active", ctypes.c_uint64),
        ("evals", ctypes.c_uint64),
        ("launches", ctypes.c_uint64),
        ("walk_launches", ctypes.c_uint64),
        ("busy_ms", ctypes.c_double),
        ("mem_used", ctypes.c_uint64),
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("evals_run", ctypes.c_uint64),
        ("mem_peak", ctypes.c_uint64),
        ("fixed_bytes", ctypes.c_uint64),
        ("lane_launches", ctypes.c_uint64),
        ("lane_unrolled_launches", ctypes.c_uint64),
        ("warp_launches", ctypes.c_uint64),
    ]


_lib = None

_EXPORTS = {
    # name: (restype, argtypes)
    "labs_opts_init": (None, [ctypes.POINTER(labs_opts)]),
    "labs_status_str": (ctypes.c_char_p, [ctypes.c_int32]),
    "labs_energy": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int32]),
    "labs_energy_batch": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_int32]),
    "labs_walks": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(labs_opts),
                                    ctypes.POINTER(labs_stats)]),
    "labs_walks_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "labs_saw_round": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32]),
    "labs_saw_round_noalloc": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                                ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "labs_batch_create": (ctypes.c_int32, [ctypes.POINTER(labs_problem), ctypes.c_int32,
                                           ctypes.POINTER(labs_batch_opts), ctypes.POINTER(ctypes.c_void_p)]),
    "labs_batch_run": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(labs_stats)]),
    "labs_batch_result": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "labs_batch_plane_steps": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]),
    "labs_batch_shape": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "labs_batch_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "labs_serve_cfg_init": (None, [ctypes.POINTER(labs_serve_cfg)]),
    "labs_serve_create": (ctypes.c_int32, [ctypes.POINTER(labs_serve_cfg), ctypes.POINTER(ctypes.c_void_p)]),
    "labs_serve_submit": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(labs_problem),
                                           ctypes.POINTER(ctypes.c_uint64)]),
    "labs_serve_poll": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(labs_result),
                                         ctypes.c_void_p]),
    "labs_serve_wait": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.POINTER(labs_result), ctypes.c_void_p]),
    "labs_serve_get_stats": (ctypes.c_int32, [ctypes.c_void_p, ctypes.POINTER(labs_serve_stats)]),
    "labs_serve_destroy": (ctypes.c_int32, [ctypes.c_void_p]),
    "labs_walks_full": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.POINTER(labs_opts), ctypes.POINTER(labs_stats)]),
    "labs_walks_full_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                         ctypes.c_int32]),
    "labs_saw_round_full": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int32,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.c_int32, ctypes.c_void_p]),
    "labs_from_hex": (ctypes.c_int32, [ctypes.c_char_p, ctypes.c_int32, ctypes.c_void_p]),
    "labs_to_hex": (ctypes.c_int32, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t]),
    "labs_model_lambda": (ctypes.c_double, [ctypes.c_int32]),
    "labs_model_nses_limit": (ctypes.c_double, [ctypes.c_int32, ctypes.c_double, ctypes.c_int32]),
    "labs_model_p_optimal": (ctypes.c_double, [ctypes.c_int32, ctypes.c_double]),
    "labs_model_nses_of_evals": (ctypes.c_double, [ctypes.c_int32, ctypes.c_uint64]),
    "labs_model_budget": (ctypes.c_uint64, [ctypes.c_int32, ctypes.c_double]),
}


def library_path() -> str:
    return LIB_PATH


def load():
    """Load liblabs_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblabs_gb300.so is not built; run `python -m paper_2210_15962_gb300.build` "
                               "(needs nvcc with sm_103a support)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _EXPORTS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_str(status: int) -> str:
    return load().labs_status_str(status).decode()


def _check(status: int, what: str):
    if status != LABS_OK:
        raise LabsError(status, what)


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a is not None else None


# --------------------------------------------- predictive model (Section 4.1, Eq. 6-7)
def labs_model_lambda(L: int) -> float:
    """lambda(L) of the run-length model (C ABI; NaN for an invalid L)."""
    return load().labs_model_lambda(L)


def labs_model_nses_limit(L: int, P: float, N: int) -> float:
    """Eq. 6: evaluations per run (the paper's count) for probability P with N runs."""
    return load().labs_model_nses_limit(L, P, N)


def labs_model_p_optimal(L: int, nses: float) -> float:
    """Eq. 7: probability of an optimum after nses evaluations (the paper's count)."""
    return load().labs_model_p_optimal(L, nses)


def labs_model_nses_of_evals(L: int, evals: int) -> float:
    """The paper's evaluation count (D - 1 per step) for this library's (D per step)."""
    return load().labs_model_nses_of_evals(L, int(evals))


def labs_model_budget(L: int, P: float) -> int:
    """Step budget (this library's evaluations) at which Eq. 7 reaches P; 0 if invalid."""
    return int(load().labs_model_budget(L, P))


def _cuda_arg(t, dtypes, numel, what, name, optional=False):
    """Device pointer of a caller-owned tensor after checking that the library
    can use it: a contiguous CUDA tensor on the current device, of one of
    `dtypes` (None: any), with at least `numel` elements.  Anything else raises
    LabsError(LABS_EINVAL) before the library is called, since the library
    cannot check a raw device pointer and would write past a short buffer."""
    import torch
    if t is None:
        if optional:
            return None
        raise LabsError(LABS_EINVAL, "%s (%s is required)" % (what, name))
    dev = torch.cuda.current_device() if torch.cuda.is_available() else None
    ok = (isinstance(t, torch.Tensor) and t.is_cuda and t.device.index == dev and t.is_contiguous()
          and (dtypes is None or t.dtype in dtypes) and t.numel() >= numel)
    if not ok:
        kind = "/".join(str(d) for d in dtypes) if dtypes else "any-type"
        raise LabsError(LABS_EINVAL, "%s (%s must be a contiguous %s CUDA tensor on the current device with at "
                                     "least %d elements)" % (what, name, kind, numel))
    return ctypes.c_void_p(t.data_ptr())


def labs_energy(seq) -> int:
    """Eq. 1 energy of one +-1 sequence (host array), computed on the GPU."""
    s = np.ascontiguousarray(seq, dtype=np.int8)
    e = load().labs_energy(_ptr(s), s.size)
    if e < 0:
        raise LabsError(int(e), "labs_energy")
    return int(e)


def labs_energy_batch(seqs, stream=None, check: bool = True):
    """Eq. 1 energies of a (n, L) int8 CUDA tensor, returned as an int64 CUDA tensor."""
    import torch
    if not (isinstance(seqs, torch.Tensor) and seqs.is_cuda and seqs.dtype == torch.int8 and seqs.dim() == 2
            and seqs.device.index == torch.cuda.current_device()):
        raise ValueError("seqs must be a 2-D int8 CUDA tensor on the current device")
    seqs = seqs.contiguous()
    out = torch.empty(seqs.shape[0], dtype=torch.int64, device=seqs.device)
    st = stream if stream is not None else torch.cuda.current_stream(seqs.device)
    _check(load().labs_energy_batch(ctypes.c_void_p(seqs.data_ptr()), seqs.shape[0], seqs.shape[1],
                                    ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(st.cuda_stream), int(check)),
           "labs_energy_batch")
    return out


def make_opts(stream=None, device_buffers=False, recheck_every=0, target_E=-1, max_rounds=0, workspace=None,
              evals_per_seed=None, rounds_per_seed=None, kernel=0) -> labs_opts:
    o = labs_opts()
    load().labs_opts_init(ctypes.byref(o))
    if stream is not None:
        o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    o.device_buffers = int(bool(device_buffers))
    o.recheck_every = int(recheck_every)
    o.target_E = int(target_E)
    o.max_rounds = int(max_rounds)
    o.kernel = int(kernel)
    if workspace is not None:
        o.workspace = _cuda_arg(workspace, None, 1, "labs_walks", "workspace")
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    if evals_per_seed is not None:
        o.evals_per_seed = ctypes.c_void_p(evals_per_seed.data_ptr() if hasattr(evals_per_seed, "data_ptr")
                                           else evals_per_seed.ctypes.data)
    if rounds_per_seed is not None:
        o.rounds_per_seed = ctypes.c_void_p(rounds_per_seed.data_ptr() if hasattr(rounds_per_seed, "data_ptr")
                                            else rounds_per_seed.ctypes.data)
    return o


SPACES = ("skew", "full")  # the skew-symmetric sequences of odd L, or all 2^L sequences


def _space(space: str) -> bool:
    if space not in SPACES:
        raise ValueError("space must be 'skew' or 'full'")
    return space == "full"


def labs_walks_workspace_size(L: int, n_seeds: int, walks_per_seed: int, walk_len: int, space: str = "skew") -> int:
    fn = load().labs_walks_full_workspace_size if _space(space) else load().labs_walks_workspace_size
    return int(fn(L, n_seeds, walks_per_seed, walk_len))


def labs_walks(L: int, seeds, walks_per_seed: int, walk_len: int, step_budget: int, *, target_E: int = -1,
               max_rounds: int = 0, recheck_every: int = 0, stream=None, workspace=None, kernel: int = 0,
               space: str = "skew") -> dict:
    """Algorithm 1 around Algorithm 2 for every seed; host buffers in and out
    (space="full": labs_walks_full over all 2^L sequences).

    Returns dict(best_seq=(n, L) int8, best_E=(n,) int64, evals=(n,) uint64,
    rounds=(n,) int32, stats=dict).
    """
    full = _space(space)
    sd = np.ascontiguousarray(np.atleast_1d(np.asarray(seeds, dtype=np.uint64)))
    n = sd.size
    best_seq = np.zeros((n, L), dtype=np.int8)
    best_E = np.zeros(n, dtype=np.int64)
    evals = np.zeros(n, dtype=np.uint64)
    rounds = np.zeros(n, dtype=np.int32)
    o = make_opts(stream=stream, recheck_every=recheck_every, target_E=target_E, max_rounds=max_rounds,
                  workspace=workspace, evals_per_seed=evals, rounds_per_seed=rounds, kernel=kernel)
    stats = labs_stats()
    fn = load().labs_walks_full if full else load().labs_walks
    _check(fn(L, _ptr(sd), n, walks_per_seed, walk_len, step_budget, _ptr(best_seq), _ptr(best_E), ctypes.byref(o),
              ctypes.byref(stats)), "labs_walks_full" if full else "labs_walks")
    return {"best_seq": best_seq, "best_E": best_E, "evals": evals, "rounds": rounds, "stats": stats.as_dict()}


def labs_walks_device(L: int, seeds, walks_per_seed: int, walk_len: int, step_budget: int, best_seq, best_E, *,
                      target_E: int = -1, max_rounds: int = 0, recheck_every: int = 0, stream=None,
                      workspace=None, evals_per_seed=None, rounds_per_seed=None, kernel: int = 0,
                      space: str = "skew") -> dict:
    """labs_walks on device-resident buffers (torch CUDA tensors): seeds int64/uint64 (n,),
    best_seq int8 (n, L), best_E int64 (n,).  Stream-ordered; returns the call's stats."""
    import torch
    full = _space(space)
    what = "labs_walks_full" if full else "labs_walks"
    n = seeds.numel() if isinstance(seeds, torch.Tensor) else 0
    if n < 1 or L < 1:
        raise LabsError(LABS_EINVAL, what)
    i64 = (torch.int64, torch.uint64) if hasattr(torch, "uint64") else (torch.int64,)
    sd = _cuda_arg(seeds, i64, n, what, "seeds")
    bs = _cuda_arg(best_seq, (torch.int8,), n * L, what, "best_seq")
    be = _cuda_arg(best_E, (torch.int64,), n, what, "best_E")
    _cuda_arg(evals_per_seed, i64, n, what, "evals_per_seed", optional=True)
    _cuda_arg(rounds_per_seed, (torch.int32,), n, what, "rounds_per_seed", optional=True)
    o = make_opts(stream=stream, device_buffers=True, recheck_every=recheck_every, target_E=target_E,
                  max_rounds=max_rounds, workspace=workspace, evals_per_seed=evals_per_seed,
                  rounds_per_seed=rounds_per_seed, kernel=kernel)
    stats = labs_stats()
    fn = load().labs_walks_full if full else load().labs_walks
    _check(fn(L, sd, n, walks_per_seed, walk_len, step_budget, bs, be, ctypes.byref(o), ctypes.byref(stats)), what)
    return stats.as_dict()


def labs_saw_round(L: int, seed: int, round_: int, n_walks: int, walk_len: int, *, recheck_every: int = 0,
                   trace_begin: int = 0, trace_count: int = 0, visited_walk: int = -1, kernel: int = 0,
                   space: str = "skew") -> dict:
    """One round of walks 0..n_walks-1 with per-walk results (and optional traces / visited keys);
    space="full" walks all 2^L sequences (labs_saw_round_full)."""
    full = _space(space)
    D = L if full else (L + 1) // 2
    best_E = np.zeros(n_walks, dtype=np.int64)
    best_seq = np.zeros((n_walks, L), dtype=np.int8)
    moves = np.zeros(n_walks, dtype=np.int32)
    stuck = np.zeros(n_walks, dtype=np.int32)
    best_step = np.zeros(n_walks, dtype=np.int32)
    trace = np.full((trace_count, walk_len), -1, dtype=np.int32) if trace_count > 0 else None
    kout = (D + 63) // 64
    vcap = walk_len + 1
    visited = np.zeros((vcap, kout), dtype=np.uint64) if visited_walk >= 0 else None
    vcount = np.zeros(1, dtype=np.int32)
    args = (L, seed, round_, n_walks, walk_len, recheck_every, _ptr(best_E), _ptr(best_seq), _ptr(moves),
            _ptr(stuck), _ptr(best_step), _ptr(trace) if trace is not None else None, trace_begin, trace_count,
            visited_walk, _ptr(visited) if visited is not None else None, vcap,
            _ptr(vcount) if visited is not None else None)
    if full:
        if kernel not in (0, 1):
            raise LabsError(LABS_EINVAL, "labs_saw_round_full")
        _check(load().labs_saw_round_full(*args), "labs_saw_round_full")
    else:
        _check(load().labs_saw_round(*args, kernel), "labs_saw_round")
    out = {"best_E": best_E, "best_seq": best_seq, "moves": moves, "stuck": stuck, "best_step": best_step}
    if trace is not None:
        out["trace"] = trace
    if visited is not None:
        out["visited"] = visited[:min(int(vcount[0]), vcap)]
        out["visited_count"] = int(vcount[0])
    return out


def labs_saw_round_noalloc(L: int, seed: int, round_: int, n_walks: int, walk_len: int, walk_best_E, walk_best_seq,
                           walk_moves=None, walk_stuck=None, stream=None) -> None:
    """labs_saw_round into caller-owned CUDA tensors, using only the library's fixed static scratch
    (for callers that may not allocate device memory; see include/labs.h).

    walk_best_E: int64 (n_walks,), walk_best_seq: int8 (n_walks, L) or (n_walks * L,), walk_moves and
    walk_stuck: int32 (n_walks,) or None; all contiguous CUDA tensors on the current device.  Anything
    else raises LabsError(LABS_EINVAL) before the library is called."""
    import torch
    what = "labs_saw_round_noalloc"
    if n_walks < 1 or L < 1:
        raise LabsError(LABS_EINVAL, what)
    args = (_cuda_arg(walk_best_E, (torch.int64,), n_walks, what, "walk_best_E"),
            _cuda_arg(walk_best_seq, (torch.int8,), n_walks * L, what, "walk_best_seq"),
            _cuda_arg(walk_moves, (torch.int32,), n_walks, what, "walk_moves", optional=True),
            _cuda_arg(walk_stuck, (torch.int32,), n_walks, what, "walk_stuck", optional=True))
    st = ctypes.c_void_p(stream.cuda_stream) if stream is not None else None
    _check(load().labs_saw_round_noalloc(L, seed, round_, n_walks, walk_len, *args, st), "labs_saw_round_noalloc")


def make_problem(L, walks, walk_len, seed, step_budget, target_E=-1) -> labs_problem:
    return labs_problem(int(L), int(walks), int(walk_len), 0, int(seed), int(step_budget), int(target_E))


class Batch:
    """labs_batch_*: many problems of uneven L solved together by the persistent batch kernel.

    problems: iterable of labs_problem or (L, walks, walk_len, seed, step_budget[, target_E]) tuples.
    """

    def __init__(self, problems, *, use_graph=False, autotune=False, block_threads=0, table_factor_x10=0,
                 rounds_per_launch=0, walk_mode=0, stream=None):
        probs = [p if isinstance(p, labs_problem) else make_problem(*p) for p in problems]
        self.problems = probs
        arr = (labs_problem * len(probs))(*probs)
        o = labs_batch_opts()
        if stream is not None:
            o.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        o.use_graph = int(bool(use_graph))
        o.autotune = int(bool(autotune))
        o.block_threads = int(block_threads)
        o.table_factor_x10 = int(table_factor_x10)
        o.rounds_per_launch = int(rounds_per_launch)
        o.walk_mode = int(walk_mode)
        h = ctypes.c_void_p()
        _check(load().labs_batch_create(arr, len(probs), ctypes.byref(o), ctypes.byref(h)), "labs_batch_create")
        self._h = h

    def run(self) -> dict:
        st = labs_stats()
        _check(load().labs_batch_run(self._h, ctypes.byref(st)), "labs_batch_run")
        return st.as_dict()

    def result(self, i: int) -> dict:
        L = self.problems[i].L
        seq = np.zeros(L, dtype=np.int8)
        E = np.zeros(1, dtype=np.int64)
        ev = np.zeros(1, dtype=np.uint64)
        rd = np.zeros(1, dtype=np.int32)
        _check(load().labs_batch_result(self._h, i, _ptr(seq), _ptr(E), _ptr(ev), _ptr(rd)), "labs_batch_result")
        ps = np.zeros(1, dtype=np.uint64)
        _check(load().labs_batch_plane_steps(self._h, i, _ptr(ps)), "labs_batch_plane_steps")
        return {"best_seq": seq, "best_E": int(E[0]), "evals": int(ev[0]), "rounds": int(rd[0]),
                "plane_steps": int(ps[0])}

    def results(self) -> list:
        return [self.result(i) for i in range(len(self.problems))]

    def shape(self, W: int) -> dict:
        v = np.zeros(5, dtype=np.int32)
        _check(load().labs_batch_shape(self._h, W, _ptr(v[0:1]), _ptr(v[1:2]), _ptr(v[2:3]), _ptr(v[3:4]),
                                       _ptr(v[4:5])), "labs_batch_shape")
        return {"block_threads": int(v[0]), "table_factor_x10": int(v[1]), "resident_walks": int(v[2]),
                "warp_per_walk": int(v[3]) == 1, "cta_per_walk": int(v[3]) == 2,
                "walk_unit": ("lane", "warp", "cta")[int(v[3])], "unroll": int(v[4])}

    def close(self):
        if getattr(self, "_h", None):
            load().labs_batch_destroy(self._h)
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


class Server:
    """labs_serve_*: a continuous-batching solve server on the current device."""

    def __init__(self, *, mem_bytes=None, max_active=None, max_L=None, max_walks=None, max_walk_len=None,
                 rounds_per_launch=None, block_threads=None, walk_mode=None, stream=None):
        c = labs_serve_cfg()
        load().labs_serve_cfg_init(ctypes.byref(c))
        for k, v in dict(mem_bytes=mem_bytes, max_active=max_active, max_L=max_L, max_walks=max_walks,
                         max_walk_len=max_walk_len, rounds_per_launch=rounds_per_launch,
                         block_threads=block_threads, walk_mode=walk_mode).items():
            if v is not None:
                setattr(c, k, int(v))
        if stream is not None:
            c.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        h = ctypes.c_void_p()
        _check(load().labs_serve_create(ctypes.byref(c), ctypes.byref(h)), "labs_serve_create")
        self._h = h
        self._L = {}

    def submit(self, L, walks, walk_len, seed, step_budget=None, target_E=-1, p_target=None) -> int:
        """Queue a request.  With p_target the step budget is the predictive
        model's (labs_model_budget: Eq. 6/7 reach p_target)."""
        if p_target is not None:
            step_budget = labs_model_budget(L, p_target)
            if step_budget == 0:
                raise LabsError(LABS_EINVAL, "labs_model_budget")
        p = make_problem(L, walks, walk_len, seed, step_budget, target_E)
        t = ctypes.c_uint64()
        _check(load().labs_serve_submit(self._h, ctypes.byref(p), ctypes.byref(t)), "labs_serve_submit")
        self._L[t.value] = L
        return t.value

    def _out(self, st, r, seq):
        d = {f[0]: getattr(r, f[0]) for f in labs_result._fields_}
        d["best_seq"] = seq
        d["latency_s"] = (r.t_done_ns - r.t_submit_ns) / 1e9 if r.t_done_ns else None
        return d

    def poll(self, ticket):
        """None while pending, else the result dict (raises on an error status)."""
        r = labs_result()
        seq = np.zeros(self._L.get(ticket, LABS_L_MAX), dtype=np.int8)
        st = load().labs_serve_poll(self._h, ticket, ctypes.byref(r), _ptr(seq))
        if st == LABS_PENDING:
            return None
        _check(st, "labs_serve_poll")
        return self._out(st, r, seq)

    def wait(self, ticket, timeout_s=600.0):
        r = labs_result()
        seq = np.zeros(self._L.get(ticket, LABS_L_MAX), dtype=np.int8)
        st = load().labs_serve_wait(self._h, ticket, int(timeout_s * 1000), ctypes.byref(r), _ptr(seq))
        _check(st, "labs_serve_wait")
        return self._out(st, r, seq)

    def stats(self) -> dict:
        s = labs_serve_stats()
        _check(load().labs_serve_get_stats(self._h, ctypes.byref(s)), "labs_serve_get_stats")
        return {f[0]: getattr(s, f[0]) for f in labs_serve_stats._fields_ if f[0] != "reserved"}

    def close(self):
        if getattr(self, "_h", None):
            load().labs_serve_destroy(self._h)
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


def to_hex(seq) -> str:
    """Table 1 code of a skew-symmetric sequence (C ABI labs_to_hex): ceil(D/4)
    upper-case hex digits of its first D values, s_1 most significant, -1 -> 1."""
    s = np.ascontiguousarray(seq, dtype=np.int8)
    out = ctypes.create_string_buffer(s.size // 8 + 8)
    _check(load().labs_to_hex(_ptr(s), s.size, out, len(out)), "labs_to_hex")
    return out.value.decode()


def from_hex(hexstr: str, L: int) -> np.ndarray:
    """The length-L skew-symmetric sequence of a Table 1 code (C ABI labs_from_hex)."""
    s = np.zeros(L, dtype=np.int8)
    st = load().labs_from_hex(hexstr.encode(), L, _ptr(s))
    if st != LABS_OK:
        raise LabsError(st, "labs_from_hex")
    return s
