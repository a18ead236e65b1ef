"""Thin Python binding of the libpdw1 C ABI (include/pdw1.h).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory and the current stream.  If the compiled
library is missing this module raises at import: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpdw1.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libpdw1.so is not built (%s); run paper_2110_14734_gb300/build.py" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)

PD_OK, PD_EINVAL, PD_ENOMEM, PD_ECUDA, PD_ETIMEOUT, PD_ECAPACITY, PD_EOVERFLOW, PD_EINFEASIBLE = range(8)
STATUS_NAMES = ["PD_OK", "PD_EINVAL", "PD_ENOMEM", "PD_ECUDA", "PD_ETIMEOUT", "PD_ECAPACITY", "PD_EOVERFLOW",
                "PD_EINFEASIBLE"]
PD_F32, PD_U8 = 0, 1


class pd_diagram(C.Structure):
    _fields_ = [("bd", C.c_void_p), ("n", C.c_int64), ("dtype", C.c_int32), ("on_host", C.c_int32)]


class pd_opts(C.Structure):
    _fields_ = [("coord_shift", C.c_int32), ("s_override", C.c_int32), ("condense", C.c_int32),
                ("perturb", C.c_int32), ("seed", C.c_uint64), ("alpha", C.c_int32), ("verify", C.c_int32),
                ("max_rounds", C.c_int64), ("time_limit_ms", C.c_int64), ("update_every", C.c_int64),
                ("seq_threshold", C.c_int32), ("solver", C.c_int32), ("ns_block", C.c_int64),
                ("ns_transport", C.c_int32), ("ns_smem", C.c_int32), ("batch_slots", C.c_int32),
                ("batch_threads", C.c_int32),
                ("nn_prune", C.c_int32), ("warm_start", C.c_int32), ("ns_walk", C.c_int32),
                ("tree", C.c_int32), ("diag_kappa", C.c_int32), ("diag_tau", C.c_int64),
                ("warm_cells", C.c_int32), ("nn_wave0", C.c_int32)]


class pd_nodes(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("X", C.c_void_p), ("Y", C.c_void_p), ("cntA", C.c_void_p),
                ("cntB", C.c_void_p), ("morton", C.c_void_p)]


class pd_network(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_arcs", C.c_int64), ("row_ptr", C.c_void_p), ("head", C.c_void_p),
                ("cost", C.c_void_p), ("supply", C.c_void_p)]


class pd_result(C.Structure):
    _fields_ = [("w1", C.c_double), ("opt_quanta", C.c_int64), ("rwmd_quanta", C.c_int64),
                ("rwmd_A", C.c_int64), ("rwmd_B", C.c_int64), ("slack_quanta", C.c_int64),
                ("mass_A", C.c_int64), ("mass_B", C.c_int64), ("s", C.c_int32), ("coord_shift", C.c_int32),
                ("delta", C.c_double), ("cell_quanta", C.c_int64), ("shift_quanta", C.c_int64),
                ("n_nodes", C.c_int64), ("n_arcs", C.c_int64), ("phases", C.c_int32), ("verified", C.c_int32),
                ("rounds", C.c_int64), ("pushes", C.c_int64), ("relabels", C.c_int64),
                ("repair_passes", C.c_int64), ("price_updates", C.c_int64), ("update_passes", C.c_int64),
                ("pivots", C.c_int64), ("degenerate", C.c_int64), ("arcs_priced", C.c_int64),
                ("solve_method", C.c_int32),
                ("cert_failures", C.c_int32), ("kernel_launches", C.c_int64), ("ns_kernel_ms", C.c_float),
                ("warm_used", C.c_int32), ("stage_ms", C.c_float * 8), ("warm_ms", C.c_float * 2),
                ("warm_pivots", C.c_int64)]

    def to_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("stage_ms", "warm_ms")}
        d["stage_ms"] = list(self.stage_ms)
        d["warm_ms"] = list(self.warm_ms)
        return d


class pd_nn_result(C.Structure):
    _fields_ = [("nn_index", C.c_int64), ("nn_opt_quanta", C.c_int64), ("nn_w1", C.c_double),
                ("solved", C.c_int64), ("pruned", C.c_int64), ("waves", C.c_int32), ("coord_shift", C.c_int32),
                ("lb_ms", C.c_float), ("solve_ms", C.c_float), ("total_ms", C.c_float), ("wcd_above", C.c_int32)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


WS_NFEAT = 72
WS_NPARAMS = 25985


class pd_ws_stats(C.Structure):
    _fields_ = [("rows", C.c_int64), ("pairs", C.c_int32), ("steps", C.c_int32), ("loss_first", C.c_float),
                ("loss_last", C.c_float), ("collect_ms", C.c_float), ("train_ms", C.c_float),
                ("cold_pivots", C.c_int64), ("val_rows", C.c_int64), ("val_pairs", C.c_int32),
                ("best_epoch", C.c_int32), ("val_loss_zero", C.c_float), ("val_loss", C.c_float)]

    def to_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib.pd_create.restype = C.c_int
_lib.pd_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]
_lib.pd_destroy.restype = None
_lib.pd_destroy.argtypes = [C.c_void_p]
_lib.pd_last_error.restype = C.c_char_p
_lib.pd_last_error.argtypes = [C.c_void_p]
_lib.pd_kernel_launches.restype = C.c_int64
_lib.pd_kernel_launches.argtypes = []
_lib.pd_opts_default.restype = None
_lib.pd_opts_default.argtypes = [C.POINTER(pd_opts)]
_lib.pd_condense.restype = C.c_int
_lib.pd_condense.argtypes = [C.c_void_p, pd_diagram, pd_diagram, C.c_int64, C.c_int64, C.POINTER(pd_opts),
                             C.POINTER(pd_nodes), C.c_void_p]
_lib.pd_rwmd_lower_bound.restype = C.c_int
_lib.pd_rwmd_lower_bound.argtypes = [C.c_void_p, pd_diagram, pd_diagram, C.POINTER(pd_opts),
                                     C.POINTER(C.c_int64), C.c_void_p]
_lib.pd_wspd_sparsify.restype = C.c_int
_lib.pd_wspd_sparsify.argtypes = [C.c_void_p, C.POINTER(pd_nodes), C.c_int32, C.POINTER(pd_network), C.c_void_p]
_lib.pd_wspd_count.restype = C.c_int
_lib.pd_wspd_count.argtypes = [C.c_void_p, C.POINTER(pd_nodes), C.c_int32, C.c_int32, C.POINTER(C.c_int64),
                               C.c_void_p]
_lib.pd_wspd_sparsify_tree.restype = C.c_int
_lib.pd_wspd_sparsify_tree.argtypes = [C.c_void_p, C.POINTER(pd_nodes), C.c_int32, C.c_int32, C.POINTER(pd_nodes),
                                       C.POINTER(pd_network), C.c_void_p]
_lib.pd_mcf_solve.restype = C.c_int
_lib.pd_mcf_solve.argtypes = [C.c_void_p, C.POINTER(pd_network), C.POINTER(pd_opts), C.POINTER(C.c_int64),
                              C.POINTER(pd_result), C.c_void_p]
_lib.pd_w1_approx.restype = C.c_int
_lib.pd_w1_approx.argtypes = [C.c_void_p, pd_diagram, pd_diagram, C.c_double, C.POINTER(pd_opts),
                              C.POINTER(pd_result), C.c_void_p]
_lib.pd_w1_sparsify_count.restype = C.c_int
_lib.pd_w1_sparsify_count.argtypes = [C.c_void_p, pd_diagram, pd_diagram, C.c_double, C.POINTER(pd_opts),
                                      C.POINTER(pd_result), C.c_void_p]
_lib.pd_w1_approx_batch.restype = C.c_int
_lib.pd_w1_approx_batch.argtypes = [C.c_void_p, C.POINTER(pd_diagram), C.POINTER(pd_diagram), C.c_int64,
                                    C.c_double, C.POINTER(pd_opts), C.POINTER(pd_result), C.c_void_p]

_lib.pd_db_build.restype = C.c_int
_lib.pd_db_build.argtypes = [C.c_void_p, C.POINTER(pd_diagram), C.c_int64, C.POINTER(pd_opts), C.c_void_p]
_lib.pd_nn_search.restype = C.c_int
_lib.pd_nn_search.argtypes = [C.c_void_p, pd_diagram, C.c_double, C.POINTER(pd_opts), C.POINTER(pd_nn_result),
                              C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_void_p]

class pd_tune_result(C.Structure):
    _fields_ = [("ns_block", C.c_int64), ("ns_walk", C.c_int32), ("size_class", C.c_int32), ("candidates", C.c_int32),
                ("pairs", C.c_int32),
                ("from_cache", C.c_int32), ("best_ms", C.c_float), ("default_ms", C.c_float)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib.pd_autotune.restype = C.c_int
_lib.pd_autotune.argtypes = [C.c_void_p, C.POINTER(pd_diagram), C.POINTER(pd_diagram), C.c_int64, C.c_double,
                             C.POINTER(pd_opts), C.c_char_p, C.POINTER(pd_tune_result), C.c_void_p]
_lib.pd_tuned_block.restype = C.c_int
_lib.pd_tuned_block.argtypes = [C.c_void_p, C.c_int64, C.POINTER(C.c_int64)]

_F32P = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_lib.pd_ws_train.restype = C.c_int
_lib.pd_ws_train.argtypes = [C.c_void_p, C.POINTER(pd_diagram), C.POINTER(pd_diagram), C.c_int64, C.c_double,
                             C.POINTER(pd_opts), C.c_int32, C.c_float, C.c_uint64, C.POINTER(pd_ws_stats), C.c_void_p]
_lib.pd_ws_get_params.restype = C.c_int
_lib.pd_ws_get_params.argtypes = [C.c_void_p, _F32P]
_lib.pd_ws_set_params.restype = C.c_int
_lib.pd_ws_set_params.argtypes = [C.c_void_p, _F32P]
_lib.pd_ws_forward.restype = C.c_int
_lib.pd_ws_forward.argtypes = [C.c_void_p, _F32P, C.c_int64, _F32P, C.c_void_p]
_lib.pd_ws_grad.restype = C.c_int
_lib.pd_ws_grad.argtypes = [C.c_void_p, _F32P, _F32P, C.c_void_p, C.c_int64, _F32P, C.POINTER(C.c_float),
                            C.c_void_p]
_lib.pd_ws_save.restype = C.c_int
_lib.pd_ws_save.argtypes = [C.c_void_p, C.c_char_p]
_lib.pd_ws_load.restype = C.c_int
_lib.pd_ws_load.argtypes = [C.c_void_p, C.c_char_p]

_lib.pd_mcf_solve_noalloc.restype = C.c_int
_lib.pd_mcf_solve_noalloc.argtypes = [C.POINTER(pd_network), C.POINTER(C.c_int64), C.c_void_p]

_cudart = None


def _memcpy_d2d(dst: int, src: int, nbytes: int, stream: int):
    """cudaMemcpyAsync from the CUDA runtime the library itself links."""
    global _cudart
    if _cudart is None:
        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                _cudart = C.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise OSError("libcudart not found")
        _cudart.cudaMemcpyAsync.restype = C.c_int
        _cudart.cudaMemcpyAsync.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int, C.c_void_p]
    if nbytes:
        r = _cudart.cudaMemcpyAsync(C.c_void_p(dst), C.c_void_p(src), nbytes, 3, C.c_void_p(stream))
        if r != 0:
            raise RuntimeError("cudaMemcpyAsync failed: %d" % r)


class PDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))
        self.status = status


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def pd_kernel_launches() -> int:
    """Kernels the library has launched in this process (all threads)."""
    return int(_lib.pd_kernel_launches())


def opts(**kw) -> pd_opts:
    o = pd_opts()
    _lib.pd_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def diagram(bd) -> tuple:
    """(pd_diagram, keepalive) from a torch tensor (cuda or cpu) or numpy array
    of shape (n, 2), float32 or uint8."""
    if isinstance(bd, np.ndarray):
        bd = torch.from_numpy(np.ascontiguousarray(bd))
    if bd.dtype == torch.float32:
        dt = PD_F32
    elif bd.dtype == torch.uint8:
        dt = PD_U8
    else:
        raise TypeError("diagram must be float32 or uint8")
    bd = bd.contiguous()
    n = bd.shape[0] if bd.dim() == 2 and bd.numel() else 0
    d = pd_diagram(C.c_void_p(bd.data_ptr() if n else 0), n, dt, 0 if bd.is_cuda else 1)
    return d, bd


class Context:
    """Owns a pd_ctx (device buffers live until close())."""

    def __init__(self, device: int = 0, arena_bytes: int = 0):
        self.ptr = C.c_void_p()
        self.device = device
        st = _lib.pd_create(C.byref(self.ptr), device, arena_bytes)
        if st != PD_OK:
            raise PDError(st, "pd_create failed")

    def check(self, st):
        if st != PD_OK:
            raise PDError(st, _lib.pd_last_error(self.ptr).decode())

    def close(self):
        if self.ptr:
            _lib.pd_destroy(self.ptr)
            self.ptr = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pd_create(device: int = 0, arena_bytes: int = 0) -> Context:
    return Context(device, arena_bytes)


def _copy_out(ptr, n, dtype, device, stream):
    t = torch.empty(max(n, 0), dtype=dtype, device=device)
    if n > 0:
        _memcpy_d2d(t.data_ptr(), ptr, n * t.element_size(), stream)
    return t


def pd_condense(ctx: Context, A, B, cell_quanta: int = 1, shift_quanta: int = 0, o: pd_opts | None = None,
                stream=None) -> dict:
    """Condensed nodes (copied into torch tensors on the context's device)."""
    da, ka = diagram(A)
    db, kb = diagram(B)
    out = pd_nodes()
    s = _stream(stream)
    ctx.check(_lib.pd_condense(ctx.ptr, da, db, cell_quanta, shift_quanta, C.byref(o) if o else None,
                               C.byref(out), C.c_void_p(s)))
    dev = torch.device("cuda", ctx.device)
    N = out.n_nodes
    res = dict(n_nodes=N, X=_copy_out(out.X, N, torch.int32, dev, s), Y=_copy_out(out.Y, N, torch.int32, dev, s),
               cntA=_copy_out(out.cntA, N, torch.int64, dev, s), cntB=_copy_out(out.cntB, N, torch.int64, dev, s),
               morton=_copy_out(out.morton, N, torch.int64, dev, s))
    return res


def pd_rwmd_lower_bound(ctx: Context, A, B, o: pd_opts | None = None, stream=None):
    da, ka = diagram(A)
    db, kb = diagram(B)
    out = (C.c_int64 * 3)()
    ctx.check(_lib.pd_rwmd_lower_bound(ctx.ptr, da, db, C.byref(o) if o else None, out,
                                       C.c_void_p(_stream(stream))))
    return int(out[0]), int(out[1]), int(out[2])


def pd_wspd_sparsify(ctx: Context, nodes: dict, s: int, stream=None) -> dict:
    """nodes: dict of cuda tensors X, Y (int32), cntA, cntB (int64), morton (int64)."""
    N = int(nodes["X"].numel())
    keep = [nodes[k].contiguous() for k in ("X", "Y", "cntA", "cntB", "morton")]
    nd = pd_nodes(N, *[C.c_void_p(t.data_ptr() if N else 0) for t in keep])
    out = pd_network()
    st = _stream(stream)
    ctx.check(_lib.pd_wspd_sparsify(ctx.ptr, C.byref(nd), int(s), C.byref(out), C.c_void_p(st)))
    dev = torch.device("cuda", ctx.device)
    n, m = out.n_nodes, out.n_arcs
    return dict(n_nodes=n, n_arcs=m, row_ptr=_copy_out(out.row_ptr, n + 1, torch.int64, dev, st),
                head=_copy_out(out.head, m, torch.int32, dev, st), cost=_copy_out(out.cost, m, torch.int64, dev, st),
                supply=_copy_out(out.supply, n, torch.int64, dev, st))


def pd_wspd_sparsify_tree(ctx: Context, nodes: dict, s: int, tree: int, stream=None) -> tuple:
    """As pd_wspd_sparsify on the radix tree (tree=0) or the paper's split tree
    (tree=1).  Returns (network dict, nodes dict in the tree's leaf order)."""
    N = int(nodes["X"].numel())
    keep = [nodes[k].contiguous() for k in ("X", "Y", "cntA", "cntB", "morton")]
    nd = pd_nodes(N, *[C.c_void_p(t.data_ptr() if N else 0) for t in keep])
    out = pd_network()
    ordered = pd_nodes()
    st = _stream(stream)
    ctx.check(_lib.pd_wspd_sparsify_tree(ctx.ptr, C.byref(nd), int(s), int(tree), C.byref(ordered), C.byref(out),
                                         C.c_void_p(st)))
    dev = torch.device("cuda", ctx.device)
    n, m = out.n_nodes, out.n_arcs
    net = dict(n_nodes=n, n_arcs=m, row_ptr=_copy_out(out.row_ptr, n + 1, torch.int64, dev, st),
               head=_copy_out(out.head, m, torch.int32, dev, st), cost=_copy_out(out.cost, m, torch.int64, dev, st),
               supply=_copy_out(out.supply, n, torch.int64, dev, st))
    nds = dict(X=_copy_out(ordered.X, N, torch.int32, dev, st), Y=_copy_out(ordered.Y, N, torch.int32, dev, st),
               cntA=_copy_out(ordered.cntA, N, torch.int64, dev, st), cntB=_copy_out(ordered.cntB, N, torch.int64, dev, st))
    return net, nds


def pd_wspd_count(ctx: Context, nodes: dict, s: int, tree: int = 0, stream=None) -> int:
    """Arcs of the sparse network over `nodes` (as pd_wspd_sparsify_tree), counted without building it."""
    N = int(nodes["X"].numel())
    keep = [nodes[k].contiguous() for k in ("X", "Y", "cntA", "cntB", "morton")]
    nd = pd_nodes(N, *[C.c_void_p(t.data_ptr() if N else 0) for t in keep])
    m = C.c_int64()
    ctx.check(_lib.pd_wspd_count(ctx.ptr, C.byref(nd), int(s), int(tree), C.byref(m), C.c_void_p(_stream(stream))))
    return int(m.value)


def pd_mcf_solve(ctx: Context, net: dict, o: pd_opts | None = None, stream=None):
    """net: dict of cuda tensors row_ptr, head, cost, supply (int64 / int32).
    Returns (OPT, stats dict)."""
    keep = [net["row_ptr"].contiguous(), net["head"].contiguous(), net["cost"].contiguous(),
            net["supply"].contiguous()]
    n = int(keep[0].numel()) - 1
    m = int(keep[1].numel())
    nw = pd_network(n, m, *[C.c_void_p(t.data_ptr()) for t in keep])
    opt = C.c_int64()
    res = pd_result()
    ctx.check(_lib.pd_mcf_solve(ctx.ptr, C.byref(nw), C.byref(o) if o else None, C.byref(opt), C.byref(res),
                                C.c_void_p(_stream(stream))))
    return int(opt.value), res.to_dict()


def pd_w1_sparsify_count(ctx: Context, A, B, eps: float, o: pd_opts | None = None, stream=None) -> dict:
    """Algorithm 4 up to the sparse network (arcs counted, nothing solved): the result dict's sizes."""
    da, ka = diagram(A)
    db, kb = diagram(B)
    res = pd_result()
    ctx.check(_lib.pd_w1_sparsify_count(ctx.ptr, da, db, float(eps), C.byref(o) if o else None, C.byref(res),
                                        C.c_void_p(_stream(stream))))
    return res.to_dict()


def pd_w1_approx(ctx: Context, A, B, eps: float, o: pd_opts | None = None, stream=None) -> dict:
    da, ka = diagram(A)
    db, kb = diagram(B)
    res = pd_result()
    ctx.check(_lib.pd_w1_approx(ctx.ptr, da, db, float(eps), C.byref(o) if o else None, C.byref(res),
                                C.c_void_p(_stream(stream))))
    return res.to_dict()


def pd_w1_approx_batch(ctx: Context, As, Bs, eps: float, o: pd_opts | None = None, stream=None) -> list:
    """W1 of the pairs (As[i], Bs[i]); one dict per pair, as pd_w1_approx."""
    if len(As) != len(Bs):
        raise ValueError("As and Bs differ in length")
    n = len(As)
    da = (pd_diagram * max(n, 1))()
    db = (pd_diagram * max(n, 1))()
    keep = []
    for i in range(n):
        da[i], ka = diagram(As[i])
        db[i], kb = diagram(Bs[i])
        keep += [ka, kb]
    res = (pd_result * max(n, 1))()
    ctx.check(_lib.pd_w1_approx_batch(ctx.ptr, da, db, n, float(eps), C.byref(o) if o else None, res,
                                      C.c_void_p(_stream(stream))))
    return [res[i].to_dict() for i in range(n)]


def pd_w1_approx_batch_raw(ctx: Context, da, db, n: int, eps: float, o, res, stream: int):
    """Allocation-free batched call for timing loops: prebuilt ctypes arrays."""
    return _lib.pd_w1_approx_batch(ctx.ptr, da, db, n, eps, C.byref(o) if o else None, res, C.c_void_p(stream))


def pd_db_build(ctx: Context, dbs, o: pd_opts | None = None, stream=None):
    """Database for pd_nn_search; the tensors stay referenced by the context
    wrapper until the next build."""
    n = len(dbs)
    arr = (pd_diagram * max(n, 1))()
    keep = []
    for i, d in enumerate(dbs):
        arr[i], k = diagram(d)
        keep.append(k)
    ctx.check(_lib.pd_db_build(ctx.ptr, arr, n, C.byref(o) if o else None, C.c_void_p(_stream(stream))))
    ctx._db_keep = keep  # the library reads these diagrams during searches


def pd_nn_search(ctx: Context, query, eps: float, o: pd_opts | None = None, stream=None) -> dict:
    """Nearest neighbour of `query` in the database: dict of pd_nn_result plus
    per-diagram `opt` (-1 where pruned), `lb` (the bound used) and `wcd` (the
    WCD bound alone) lists."""
    dq, kq = diagram(query)
    n = len(getattr(ctx, "_db_keep", []))
    res = pd_nn_result()
    opt = (C.c_int64 * max(n, 1))()
    lb = (C.c_int64 * max(n, 1))()
    wcd = (C.c_int64 * max(n, 1))()
    ctx.check(_lib.pd_nn_search(ctx.ptr, dq, float(eps), C.byref(o) if o else None, C.byref(res), opt, lb, wcd,
                                C.c_void_p(_stream(stream))))
    d = res.to_dict()
    d["opt"] = [int(opt[i]) for i in range(n)]
    d["lb"] = [int(lb[i]) for i in range(n)]
    d["wcd"] = [int(wcd[i]) for i in range(n)]
    return d


def pd_autotune(ctx: Context, As, Bs, eps: float, o: pd_opts | None = None, cache_path: str | None = None,
                stream=None) -> dict:
    """Time the simplex's pricing block on the sample pairs; the context keeps the best per size class."""
    n = len(As)
    da = (pd_diagram * max(n, 1))()
    db = (pd_diagram * max(n, 1))()
    keep = []
    for i in range(n):
        da[i], ka = diagram(As[i])
        db[i], kb = diagram(Bs[i])
        keep += [ka, kb]
    res = pd_tune_result()
    ctx.check(_lib.pd_autotune(ctx.ptr, da, db, n, float(eps), C.byref(o) if o else None,
                               cache_path.encode() if cache_path else None, C.byref(res), C.c_void_p(_stream(stream))))
    return res.to_dict()


def pd_tuned_block(ctx: Context, arcs_and_nodes: int) -> int:
    b = C.c_int64()
    ctx.check(_lib.pd_tuned_block(ctx.ptr, int(arcs_and_nodes), C.byref(b)))
    return int(b.value)


def pd_ws_train(ctx: Context, As, Bs, eps: float, o: pd_opts | None = None, epochs: int = 20, lr: float = 1e-3,
                seed: int = 0, stream=None) -> dict:
    """Train the context's warm-start network on cold solves of the pairs."""
    n = len(As)
    da = (pd_diagram * max(n, 1))()
    db = (pd_diagram * max(n, 1))()
    keep = []
    for i in range(n):
        da[i], ka = diagram(As[i])
        db[i], kb = diagram(Bs[i])
        keep += [ka, kb]
    st = pd_ws_stats()
    ctx.check(_lib.pd_ws_train(ctx.ptr, da, db, n, float(eps), C.byref(o) if o else None, int(epochs), float(lr),
                               int(seed), C.byref(st), C.c_void_p(_stream(stream))))
    return st.to_dict()


def pd_ws_get_params(ctx: Context) -> np.ndarray:
    p = np.zeros(WS_NPARAMS, np.float32)
    ctx.check(_lib.pd_ws_get_params(ctx.ptr, p))
    return p


def pd_ws_set_params(ctx: Context, p) -> None:
    ctx.check(_lib.pd_ws_set_params(ctx.ptr, np.ascontiguousarray(p, np.float32)))


def pd_ws_forward(ctx: Context, feats) -> np.ndarray:
    f = np.ascontiguousarray(feats, np.float32).reshape(-1, WS_NFEAT)
    y = np.zeros(len(f), np.float32)
    ctx.check(_lib.pd_ws_forward(ctx.ptr, f, len(f), y, C.c_void_p(_stream(None))))
    return y


def pd_ws_grad(ctx: Context, feats, target, mask=None):
    """(loss, gradient of the master parameters) on the device."""
    f = np.ascontiguousarray(feats, np.float32).reshape(-1, WS_NFEAT)
    t = np.ascontiguousarray(target, np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, np.float32)
    g = np.zeros(WS_NPARAMS, np.float32)
    loss = C.c_float()
    ctx.check(_lib.pd_ws_grad(ctx.ptr, f, t, m.ctypes.data_as(C.c_void_p) if m is not None else None, len(f), g,
                              C.byref(loss), C.c_void_p(_stream(None))))
    return float(loss.value), g


def pd_ws_save(ctx: Context, path: str) -> None:
    ctx.check(_lib.pd_ws_save(ctx.ptr, path.encode()))


def pd_ws_load(ctx: Context, path: str) -> None:
    ctx.check(_lib.pd_ws_load(ctx.ptr, path.encode()))


def pd_w1_approx_raw(ctx: Context, da: pd_diagram, db: pd_diagram, eps: float, o, res: pd_result, stream: int):
    """Allocation-free call for timing loops: prebuilt structs, result in res."""
    return _lib.pd_w1_approx(ctx.ptr, da, db, eps, C.byref(o) if o else None, C.byref(res), C.c_void_p(stream))


def pd_mcf_solve_noalloc(net: dict, stream=None) -> int:
    """The allocation-free solve (no context, fixed scratch in the library).
    net: dict of cuda tensors row_ptr, head, cost, supply.  Returns OPT."""
    keep = [net["row_ptr"].contiguous(), net["head"].contiguous(), net["cost"].contiguous(),
            net["supply"].contiguous()]
    n = int(keep[0].numel()) - 1
    m = int(keep[1].numel())
    nw = pd_network(n, m, *[C.c_void_p(t.data_ptr()) for t in keep])
    opt = C.c_int64()
    st = _lib.pd_mcf_solve_noalloc(C.byref(nw), C.byref(opt), C.c_void_p(_stream(stream)))
    if st != PD_OK:
        raise PDError(st, "pd_mcf_solve_noalloc failed")
    return int(opt.value)
