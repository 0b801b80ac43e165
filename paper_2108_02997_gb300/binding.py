"""Python binding of ``libpagerank.so`` (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/pagerank.h``
under the same name; all PageRank arithmetic runs in the library's CUDA
kernels. There is no CPU fallback: if the library cannot be loaded, or no
CUDA device is present, calls raise.

Low level: ``lib()`` returns the ``ctypes.CDLL`` with typed entry points and
the ``pr_options`` / ``pr_instance`` structures.

High level: :class:`Graph` owns a ``pr_graph`` handle; :func:`pr_solve` and
:func:`pr_solve_batch` accept numpy arrays (host buffers) or torch CUDA tensors
(device buffers).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import _build

PR_OK, PR_EINVAL, PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_ESTATE, PR_ENOTSUP = range(7)
PR_NORM_L1, PR_NORM_L2, PR_NORM_LINF = 1, 2, 3
PR_PREC_DF64, PR_PREC_FP64, PR_PREC_MIXED, PR_PREC_FP32, PR_PREC_AUTO = 0, 1, 2, 3, 4
PR_INIT_UNIFORM, PR_INIT_USER, PR_INIT_LEARNED, PR_INIT_CHAIN, PR_INIT_AUTO = 0, 1, 2, 3, 4
PR_LOOP_GRAPH, PR_LOOP_HOST, PR_LOOP_PERSISTENT, PR_LOOP_AUTO = 0, 1, 2, 3
LOOPS = {"graph": PR_LOOP_GRAPH, "host": PR_LOOP_HOST, "persistent": PR_LOOP_PERSISTENT, "auto": PR_LOOP_AUTO}
PR_GROUP_AUTO, PR_GROUP_PACK, PR_GROUP_SINGLE = 0, 1, 2
GROUPS = {"auto": PR_GROUP_AUTO, "pack": PR_GROUP_PACK, "single": PR_GROUP_SINGLE}
PR_KERNELS_AUTO, PR_KERNELS_FUSED, PR_KERNELS_SPLIT = 0, 1, 2
KERNELS = {"auto": PR_KERNELS_AUTO, "fused": PR_KERNELS_FUSED, "split": PR_KERNELS_SPLIT}
PRECISIONS = {"df64": PR_PREC_DF64, "fp64": PR_PREC_FP64, "mixed": PR_PREC_MIXED, "fp32": PR_PREC_FP32,
              "auto": PR_PREC_AUTO}
NORMS = {"L1": 1, "L2": 2, "Linf": 3, 1: 1, 2: 2, 3: 3}
MLP_PARAMS = 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1


class pr_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("init", C.c_int32), ("init_vec", C.c_void_p),
                ("init_on_device", C.c_int32), ("outputs_on_device", C.c_int32),
                ("switch_tol", C.c_double), ("stream", C.c_void_p),
                ("share_trajectories", C.c_int32), ("loop", C.c_int32), ("mlp", C.c_void_p),
                ("err_history", C.c_void_p), ("group", C.c_int32), ("max_passes", C.c_int32),
                ("kernels", C.c_int32), ("persist_wait_us", C.c_int32), ("reserved", C.c_int32 * 4)]


class pr_instance(C.Structure):
    _fields_ = [("g", C.c_void_p), ("alpha", C.c_double), ("tol", C.c_double), ("norm", C.c_int32),
                ("max_iter", C.c_int32), ("ranks_out", C.c_void_p), ("init_vec", C.c_void_p),
                ("iters", C.c_int32), ("converged", C.c_int32), ("err", C.c_double),
                ("err_l1", C.c_double), ("status", C.c_int32), ("reserved", C.c_int32)]


class PageRankError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({_STATUS.get(status, '?')}): {msg}")
        self.status = status


_STATUS = {0: "PR_OK", 1: "PR_EINVAL", 2: "PR_ENOMEM", 3: "PR_ECUDA", 4: "PR_ETIMEOUT", 5: "PR_ESTATE",
           6: "PR_ENOTSUP"}

# Exported symbols and their (argtypes, restype); mirrors include/pagerank.h.
_vp, _i32, _i64, _d, _f = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_float
SIGNATURES = {
    "pr_options_default": ([_vp], None),
    "pr_graph_create": ([_i32, _i64, _vp, _vp, _vp, C.POINTER(_vp)], _i32),
    "pr_graph_destroy": ([_vp], _i32),
    "pr_graph_info": ([_vp, _vp, _vp, _vp], _i32),
    "pr_solve": ([_vp, _d, _d, _i32, _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "pr_solve_batch": ([_vp, _i32, _vp], _i32),
    "pr_mlp_create": ([_vp, C.POINTER(_vp)], _i32),
    "pr_mlp_destroy": ([_vp], _i32),
    "pr_mlp_get_params": ([_vp, _vp], _i32),
    "pr_features": ([_vp, _d, _vp, _vp], _i32),
    "pr_mlp_warm_start": ([_vp, _vp, _d, _vp, _vp], _i32),
    "pr_mlp_train": ([_vp, _vp, _vp, _vp, _i32, _i32, _f, _vp, _vp], _i32),
    "pr_mlp_loss_grad": ([_vp, _vp, _d, _vp, _vp, _vp, _vp], _i32),
    "pr_last_solve_stats": ([_vp, _vp, _vp, _vp], _i32),
    "pr_last_solve_kernel_ms": ([_vp, _vp], _i32),
    "pr_last_solve_columns": ([_vp, _vp, _vp], _i32),
    "pr_last_solve_loops": ([_vp, _vp, _vp], _i32),
    "pr_test_hold_decisions": ([_i32], _i32),
    "pr_mlp_gain": ([_vp, _vp, _vp], _i32),
    "pr_mlp_set_gain": ([_vp, _d], _i32),
    "pr_graph_tune": ([_vp, _i32, _i32, _vp, _vp], _i32),
    "pr_kernel_occupancy": ([_i32, _i32, _vp], _i32),
    "pr_plan_columns": ([_i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "pr_plan_columns_shared": ([_i32, _vp, _vp, _d, _vp, _vp, _vp], _i32),
    "pr_solve_noalloc": ([_vp, _d, _d, _i32, _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "pr_workspace_info": ([_vp, _vp, _vp], _i32),
    "pr_workspace_release": ([], _i32),
    "pr_last_error": ([], C.c_char_p),
    "pr_status_string": ([_i32], C.c_char_p),
    "pr_version": ([], _i32),
}

_lib = None


def lib(build: bool = True) -> C.CDLL:
    """Load (building first if needed) libpagerank.so with typed entry points."""
    global _lib
    if _lib is None:
        so = _build.build_pagerank() if build else _build.PAGERANK_SO
        if not so.exists():
            raise RuntimeError(f"{so} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(str(so))
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != PR_OK:
        raise PageRankError(st, where, lib().pr_last_error().decode())


def default_options(**kw) -> pr_options:
    o = pr_options()
    lib().pr_options_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def current_stream_ptr() -> int:
    import torch
    return int(torch.cuda.current_stream().cuda_stream)


def _ptr_of(buf):
    """(address, on_device) of a numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("buffers must be contiguous")
        return buf.ctypes.data, False
    import torch
    if isinstance(buf, torch.Tensor):
        if not buf.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return buf.data_ptr(), buf.is_cuda
    raise TypeError(f"unsupported buffer type {type(buf)}")


class Graph:
    """A ``pr_graph`` handle built from an in-edge CSR (host arrays)."""

    def __init__(self, offsets, sources, outdeg):
        off = np.ascontiguousarray(offsets, dtype=np.int32)
        src = np.ascontiguousarray(sources, dtype=np.int32)
        od = np.ascontiguousarray(outdeg, dtype=np.int32)
        h = C.c_void_p()
        st = lib().pr_graph_create(od.shape[0], src.shape[0], off.ctypes.data,
                                   src.ctypes.data if src.size else None, od.ctypes.data, C.byref(h))
        _check(st, "pr_graph_create")
        self.handle = h
        self.n = int(od.shape[0])
        self.nnz = int(src.shape[0])

    @classmethod
    def from_csr(cls, g) -> "Graph":
        return cls(g.offsets, g.sources, g.outdeg)

    def info(self):
        n, nnz, nd = C.c_int32(), C.c_int64(), C.c_int32()
        _check(lib().pr_graph_info(self.handle, C.byref(n), C.byref(nnz), C.byref(nd)), "pr_graph_info")
        return n.value, nnz.value, nd.value

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().pr_graph_destroy(self.handle), "pr_graph_destroy")
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


@dataclass
class SolveResult:
    ranks: object
    iters: int
    err: float
    converged: bool
    err_history: np.ndarray | None = None


def _make_options(precision="df64", init=None, loop="auto", stream=None, share=True, switch_tol=1e-6,
                  outputs_on_device=False, mlp=None, group="auto", max_passes=0, kernels="auto", persist_wait_us=0):
    o = default_options()
    o.persist_wait_us = int(persist_wait_us)
    o.kernels = KERNELS[kernels] if isinstance(kernels, str) else int(kernels)
    o.group = GROUPS[group] if isinstance(group, str) else int(group)
    o.max_passes = int(max_passes)
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    if loop not in LOOPS:
        raise ValueError(f"loop must be one of {sorted(LOOPS)}")
    o.loop = LOOPS[loop]
    o.share_trajectories = 1 if share else 0
    o.switch_tol = switch_tol
    o.outputs_on_device = 1 if outputs_on_device else 0
    o.stream = stream
    keep = []
    if init is not None and not (isinstance(init, str)):
        addr, dev = _ptr_of(init)
        o.init = PR_INIT_USER
        o.init_vec = addr
        o.init_on_device = 1 if dev else 0
        keep.append(init)
    elif init in ("learned", "auto"):
        o.init = PR_INIT_LEARNED if init == "learned" else PR_INIT_AUTO
        o.mlp = mlp.handle if mlp is not None else None
    elif init == "chain":
        o.init = PR_INIT_CHAIN
    elif init is not None:
        raise ValueError(f"unknown start {init!r}")
    return o, keep


def pr_solve(g: Graph, alpha: float, tol: float, norm=PR_NORM_L1, max_iter: int = 500, *,
             precision="df64", init=None, out=None, loop="auto", stream=None, history=False,
             switch_tol=1e-6, mlp=None, kernels="auto") -> SolveResult:
    """Solve one instance. ``out``: numpy array (host) or torch CUDA tensor
    (device) of n float64; allocated as numpy when omitted."""
    if out is None:
        out = np.empty(g.n, np.float64)
    addr, dev = _ptr_of(out)
    if stream is None and dev:
        stream = current_stream_ptr()
    o, keep = _make_options(precision, init, loop, stream, True, switch_tol, dev, mlp, kernels=kernels)
    hist = np.zeros((max_iter, 3), np.float64) if history else None
    if hist is not None:
        o.err_history = hist.ctypes.data
    it, err, conv = C.c_int32(), C.c_double(), C.c_int32()
    st = lib().pr_solve(g.handle, float(alpha), float(tol), int(NORMS[norm]), int(max_iter), C.byref(o),
                        addr, C.byref(it), C.byref(err), C.byref(conv))
    _check(st, "pr_solve")
    del keep
    return SolveResult(out, it.value, err.value, bool(conv.value),
                       hist[: it.value] if hist is not None else None)


@dataclass
class Instance:
    graph: Graph
    alpha: float
    tol: float
    norm: int = PR_NORM_L1
    max_iter: int = 500
    out: object = None
    init: object = None
    iters: int = 0
    err: float = 0.0
    err_l1: float = 0.0
    converged: bool = False
    status: int = 0


# pr_instance as a numpy record (same layout), so that large batches are
# marshalled with array operations instead of one ctypes structure per instance
_INST_DTYPE = np.dtype({"names": ["g", "alpha", "tol", "norm", "max_iter", "ranks_out", "init_vec", "iters",
                                  "converged", "err", "err_l1", "status", "reserved"],
                        "formats": [np.uint64, np.float64, np.float64, np.int32, np.int32, np.uint64, np.uint64,
                                    np.int32, np.int32, np.float64, np.float64, np.int32, np.int32],
                        "offsets": [0, 8, 16, 24, 28, 32, 40, 48, 52, 56, 64, 72, 76], "itemsize": 80})
assert _INST_DTYPE.itemsize == C.sizeof(pr_instance)
for _f, *_ in pr_instance._fields_:
    assert _INST_DTYPE.fields[_f][1] == getattr(pr_instance, _f).offset, _f


class PreparedBatch:
    """A batch of :class:`Instance` marshalled once into the library's
    ``pr_instance`` array, to be solved any number of times (repeated sweeps
    over the same graphs and outputs pay no per-instance Python work per call).
    ``out`` buffers are allocated here when missing (numpy, or torch CUDA
    tensors when ``outputs_on_device``). After :meth:`solve` the results are
    numpy arrays in instance order: ``iters``, ``err``, ``err_l1``,
    ``converged``, ``status``; :meth:`fill` copies them into the instances."""

    def __init__(self, insts, outputs_on_device=False):
        n = len(insts)
        self.insts = list(insts)
        self.outputs_on_device = bool(outputs_on_device)
        arr = np.zeros(max(n, 1), _INST_DTYPE)
        self._keep = []
        if outputs_on_device:
            import torch
            for x in insts:
                if x.out is None:
                    x.out = torch.empty(x.graph.n, dtype=torch.float64, device="cuda")
                if not (isinstance(x.out, torch.Tensor) and x.out.is_cuda and x.out.is_contiguous()):
                    raise ValueError("every out must be a contiguous CUDA tensor when outputs_on_device")
            arr["ranks_out"][:n] = [x.out.data_ptr() for x in insts]
        else:
            outs = []
            for x in insts:
                if x.out is None:
                    x.out = np.empty(x.graph.n, np.float64)
                addr, dev = _ptr_of(x.out)
                if dev:
                    raise ValueError("every out must live on the device iff outputs_on_device")
                outs.append(addr)
            arr["ranks_out"][:n] = outs
        arr["g"][:n] = [x.graph.handle.value or 0 for x in insts]
        arr["alpha"][:n] = [x.alpha for x in insts]
        arr["tol"][:n] = [x.tol for x in insts]
        arr["norm"][:n] = [NORMS[x.norm] for x in insts]
        arr["max_iter"][:n] = [x.max_iter for x in insts]
        self.has_init = any(x.init is not None for x in insts)
        if self.has_init:
            inits = []
            for x in insts:
                if x.init is not None:
                    inits.append(_ptr_of(x.init)[0])
                    self._keep.append(x.init)
                else:
                    inits.append(0)
            arr["init_vec"][:n] = inits
        self.arr = arr
        self.n = n
        self._opts = {}
        self._arr_ptr = arr.ctypes.data

    def solve(self, *, precision="df64", init=None, loop="auto", stream=None, share=True, switch_tol=1e-6,
              mlp=None, check=True, group="auto", max_passes=0, kernels="auto", persist_wait_us=0):
        """One pr_solve_batch call over the prepared instances; returns its status."""
        if stream is None and self.outputs_on_device:
            stream = current_stream_ptr()
        # the options of repeated calls with the same arguments are built once
        key = None
        if init is None or isinstance(init, str):
            key = (precision, init, loop, stream, share, switch_tol, mlp.handle.value if mlp is not None else None,
                   group, max_passes, kernels, persist_wait_us)
        o = self._opts.get(key) if key is not None else None
        if o is None:
            o, keep2 = _make_options(precision, init, loop, stream, share, switch_tol, self.outputs_on_device, mlp,
                                     group, max_passes, kernels, persist_wait_us)
            if self.has_init and o.init == PR_INIT_UNIFORM:
                o.init = PR_INIT_USER
            if key is not None:
                self._opts[key] = o
        st = lib().pr_solve_batch(self._arr_ptr, self.n, C.byref(o))
        if check:
            _check(st, "pr_solve_batch")
        return st

    @property
    def iters(self):
        return self.arr["iters"][:self.n]

    @property
    def err(self):
        return self.arr["err"][:self.n]

    @property
    def err_l1(self):
        return self.arr["err_l1"][:self.n]

    @property
    def converged(self):
        return self.arr["converged"][:self.n].astype(bool)

    @property
    def status(self):
        return self.arr["status"][:self.n]

    def fill(self):
        """Copy the last call's results into the instances; returns them."""
        iters, conv, err, err1, stat = (self.arr["iters"].tolist(), self.arr["converged"].tolist(),
                                        self.arr["err"].tolist(), self.arr["err_l1"].tolist(),
                                        self.arr["status"].tolist())
        for i, x in enumerate(self.insts):
            x.iters = iters[i]
            x.err = err[i]
            x.err_l1 = err1[i]
            x.converged = bool(conv[i])
            x.status = stat[i]
        return self.insts


def pr_solve_batch(insts, *, precision="df64", init=None, loop="auto", stream=None, share=True,
                   switch_tol=1e-6, outputs_on_device=False, mlp=None, check=True, group="auto", max_passes=0,
                   kernels="auto", persist_wait_us=0):
    """Solve many instances together. Fills ``out`` (allocated as numpy, or as
    torch CUDA tensors when ``outputs_on_device``), ``iters``, ``err``,
    ``converged`` and ``status`` of every :class:`Instance`; returns the
    library status."""
    pb = PreparedBatch(insts, outputs_on_device)
    st = pb.solve(precision=precision, init=init, loop=loop, stream=stream, share=share, switch_tol=switch_tol,
                  mlp=mlp, check=False, group=group, max_passes=max_passes, kernels=kernels,
                  persist_wait_us=persist_wait_us)
    pb.fill()
    if check:
        _check(st, "pr_solve_batch")
    return st


def hold_decisions(on: bool) -> None:
    """Test hook (pr_test_hold_decisions): while on, the CTAs of persistent
    passes never announce the end of a pass, so their bounded waits run out
    (PR_ETIMEOUT)."""
    _check(lib().pr_test_hold_decisions(1 if on else 0), "pr_test_hold_decisions")


def pr_graph_tune(g: "Graph", precision="df64", max_width: int = 32, stream=None):
    """Launch times (microseconds) of the iteration kernel on ``g`` for widths
    1, 2, 4, 8, 16, 32 (0 = not measured); measured once per graph signature."""
    us = (C.c_double * 6)()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().pr_graph_tune(g.handle, p, int(max_width), stream, us), "pr_graph_tune")
    return list(us)


def kernel_occupancy(precision="df64", width: int = 1) -> int:
    """Resident CTAs per SM of the iteration kernel (needs a GPU)."""
    c = C.c_int32()
    p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().pr_kernel_occupancy(p, int(width), C.byref(c)), "pr_kernel_occupancy")
    return c.value


def plan_columns(iters, us_per_launch):
    """The PR_GROUP_AUTO planner on host data: (job_of, width_of, cost)."""
    it = np.ascontiguousarray(iters, np.float64)
    us = np.ascontiguousarray(us_per_launch, np.float64)
    if us.size != 6:
        raise ValueError("need 6 launch times (W = 1 .. 32)")
    job = np.empty(it.size, np.int32)
    wid = np.empty(it.size, np.int32)
    cost = C.c_double()
    _check(lib().pr_plan_columns(it.size, it.ctypes.data, us.ctypes.data, job.ctypes.data, wid.ctypes.data,
                                 C.byref(cost)), "pr_plan_columns")
    return job, wid, cost.value


def plan_columns_shared(iters, us_per_launch, latency_us):
    """The planner with the launch latency that jobs of one width share:
    (job_of, width_of, cost under the shared-latency model)."""
    it = np.ascontiguousarray(iters, np.float64)
    us = np.ascontiguousarray(us_per_launch, np.float64)
    if us.size != 6:
        raise ValueError("need 6 launch times (W = 1 .. 32)")
    job = np.empty(it.size, np.int32)
    wid = np.empty(it.size, np.int32)
    cost = C.c_double()
    _check(lib().pr_plan_columns_shared(it.size, it.ctypes.data, us.ctypes.data, float(latency_us), job.ctypes.data,
                                        wid.ctypes.data, C.byref(cost)), "pr_plan_columns_shared")
    return job, wid, cost.value


def workspace_info():
    """(reserved, used, used_high) bytes of the current device's workspace pool."""
    r, u, h = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().pr_workspace_info(C.byref(r), C.byref(u), C.byref(h)), "pr_workspace_info")
    return r.value, u.value, h.value


def workspace_release():
    """Return the workspace pool's unused reserved memory to the device."""
    _check(lib().pr_workspace_release(), "pr_workspace_release")


def pr_last_solve_stats():
    la, pa, km, tm = C.c_int32(), C.c_int32(), C.c_double(), C.c_double()
    lib().pr_last_solve_stats(C.byref(la), C.byref(pa), C.byref(km), C.byref(tm))
    gm, um = C.c_double(), C.c_double()
    lib().pr_last_solve_kernel_ms(C.byref(gm), C.byref(um))
    co, mc, lc = C.c_int32(), C.c_int32(), C.c_int32()
    lib().pr_last_solve_columns(C.byref(co), C.byref(mc), C.byref(lc))
    lg, lh, lp = C.c_int32(), C.c_int32(), C.c_int32()
    lib().pr_last_solve_loops(C.byref(lg), C.byref(lh), C.byref(lp))
    return {"launches": la.value, "passes": pa.value, "kernel_ms": km.value, "total_ms": tm.value,
            "gather_ms": gm.value, "update_ms": um.value, "columns": co.value, "mixed_columns": mc.value,
            "learned_columns": lc.value,
            "loop_phases": {"graph": lg.value, "host": lh.value, "persistent": lp.value}}


class MLP:
    """A ``pr_mlp`` handle: the learned warm start (5-64-64-1 GELU MLP)."""

    def __init__(self, params):
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if p.size != MLP_PARAMS:
            raise ValueError(f"need {MLP_PARAMS} parameters")
        h = C.c_void_p()
        _check(lib().pr_mlp_create(p.ctypes.data, C.byref(h)), "pr_mlp_create")
        self.handle = h

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        _check(lib().pr_mlp_get_params(self.handle, out.ctypes.data), "pr_mlp_get_params")
        return out

    def warm_start(self, g: "Graph", alpha: float, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        if stream is None:
            stream = current_stream_ptr()
        _check(lib().pr_mlp_warm_start(self.handle, g.handle, float(alpha), out.data_ptr(), stream),
               "pr_mlp_warm_start")
        return out

    def loss_grad(self, g: "Graph", alpha: float, target_r, stream=None):
        """(loss, gradient) on one set; target_r: torch CUDA float64 tensor (caller order)."""
        if stream is None:
            stream = current_stream_ptr()
        loss = C.c_float()
        grad = np.empty(MLP_PARAMS, np.float32)
        _check(lib().pr_mlp_loss_grad(self.handle, g.handle, float(alpha), target_r.data_ptr(), C.byref(loss),
                                      grad.ctypes.data, stream), "pr_mlp_loss_grad")
        return float(loss.value), grad

    def train(self, sets, epochs: int, lr: float, stream=None) -> float:
        """sets: list of (Graph, alpha, target_r CUDA float64 tensor). Returns
        the mean loss of the last epoch."""
        if stream is None:
            stream = current_stream_ptr()
        n = len(sets)
        gs = (C.c_void_p * n)(*[s[0].handle.value for s in sets])
        al = (C.c_double * n)(*[float(s[1]) for s in sets])
        tg = (C.c_void_p * n)(*[s[2].data_ptr() for s in sets])
        loss = C.c_float()
        _check(lib().pr_mlp_train(self.handle, gs, al, tg, n, int(epochs), float(lr), C.byref(loss), stream),
               "pr_mlp_train")
        return float(loss.value)

    def gain(self):
        """(gain, known): e-folds of start error the network removes (pr_mlp_gain)."""
        g, k = C.c_double(), C.c_int32()
        _check(lib().pr_mlp_gain(self.handle, C.byref(g), C.byref(k)), "pr_mlp_gain")
        return g.value, bool(k.value)

    def set_gain(self, gain: float):
        _check(lib().pr_mlp_set_gain(self.handle, float(gain)), "pr_mlp_set_gain")

    def close(self):
        if self.handle is not None and self.handle.value:
            _check(lib().pr_mlp_destroy(self.handle), "pr_mlp_destroy")
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pr_features(g: "Graph", alpha: float, out=None, stream=None):
    """(n, 5) float32 features on the device, caller order."""
    import torch
    if out is None:
        out = torch.empty((g.n, 5), dtype=torch.float32, device="cuda")
    if stream is None:
        stream = current_stream_ptr()
    _check(lib().pr_features(g.handle, float(alpha), out.data_ptr(), stream), "pr_features")
    return out


def init_mlp_params(seed: int = 7) -> np.ndarray:
    """Seeded initial parameters: weights N(0, 1/fan_in) from the counter-based
    generator, zero biases."""
    from . import graphgen
    z = graphgen.normal(seed, 9, MLP_PARAMS)
    p = np.zeros(MLP_PARAMS, np.float64)
    o = 0
    for shape, fan_in in (((64, 5), 5), ((64,), 0), ((64, 64), 64), ((64,), 0), ((1, 64), 64), ((1,), 0)):
        k = int(np.prod(shape))
        if fan_in:
            p[o:o + k] = z[o:o + k] / np.sqrt(fan_in)
        o += k
    return p.astype(np.float32)
