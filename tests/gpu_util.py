"""Helpers of the GPU parity tests (marshal a workloads.Instance through the
C ABI and bring the results back)."""
import numpy as np
import torch

from paper_2409_03686_gb300 import build as B
from paper_2409_03686_gb300 import wos

_ctx = None


def ctx():
    global _ctx
    if _ctx is None:
        B.build()
        _ctx = wos.Context(0)
    return _ctx


def gpu_build(inst, trace=True, trace_steps=False, trace_x=False, **kw):
    """Run wos_build_operator for `inst`; returns dict of numpy results."""
    dev = torch.device("cuda:0")
    pts = torch.as_tensor(inst.points, dtype=torch.float64, device=dev)
    k0 = kw.pop("k0", 0)
    k1 = kw.pop("k1", 0) or inst.N
    n = k1 - k0
    tr = torch.full((inst.M_D, n), -2, dtype=torch.int32, device=dev) if trace else None
    ts = torch.zeros((inst.M_D, n), dtype=torch.int32, device=dev) if trace_steps else None
    tx = torch.zeros((inst.M_D, n, inst.dim), dtype=torch.float64, device=dev) if trace_x else None
    counts = kw.pop("counts", None)
    unterm = kw.pop("unterminated", None)
    opts = wos.make_opts(precision=1 if inst.fp64 else 0, stream_id=inst.stream,
                         step_cap=inst.step_cap if inst.step_cap != 1_000_000 else 0,
                         k0=k0, k1=k1 if k1 != inst.N or k0 else 0,
                         trace_elem=tr, trace_steps=ts, trace_x=tx,
                         mapped=getattr(inst, "mapped", False), **kw)
    c, u, st = wos.wos_build_operator(ctx(), inst.domain, inst.K, pts, inst.partition,
                                      inst.N, inst.eps, inst.seed, opts=opts,
                                      counts=counts, unterminated=unterm)
    torch.cuda.synchronize()
    out = dict(counts=c.cpu().numpy().astype(np.int64),
               unterm=u.cpu().numpy().astype(np.int64), stats=st, counts_t=c, unterm_t=u)
    if trace:
        out["trace"] = tr.cpu().numpy()
    if trace_steps:
        out["steps"] = ts.cpu().numpy()
    if trace_x:
        out["x"] = tx.cpu().numpy()
    return out


def oracle_walks(inst, rows=None, k0=0, k1=None):
    from oracle import oracle as O
    k1 = inst.N if k1 is None else k1
    rows = np.arange(inst.M_D) if rows is None else np.asarray(rows)
    i = np.repeat(rows, k1 - k0)
    k = np.tile(np.arange(k0, k1), len(rows))
    xe, el, ns = O.walks(inst, i, k)
    shape = (len(rows), k1 - k0)
    return el.reshape(shape), ns.reshape(shape), xe.reshape(shape + (inst.dim,))
