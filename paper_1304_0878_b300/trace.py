"""Analysis of an execution trace (Context.trace_start / trace_read): one
record per finished work item with its task, item, SM, kind, and start and
end on the device's global nanosecond timer.

`summary` answers where a launch's time went: the makespan, how busy the
CTAs were, each task kind's share of the CTA time, the critical path (the
longest chain of task spans along the dependency edges), and whether any
task started before one of its predecessors ended.
"""
import numpy as np

from . import _lib

KIND_NAMES = {getattr(_lib, n): n for n in (
    "NOOP", "SCAL_F32", "POTRF", "TRSM", "SYRK", "GEMM", "POTRF_MX", "TRSM_MX", "SYRK_MX", "GEMM_MX", "QUANT",
    "TRSV_L", "GEMV_L", "TRSV_LT", "GEMV_LT", "AXPY", "RESID", "NRM", "POTRF_D", "PANEL_TRSM", "PANEL_UPD",
    "CVT", "TRTRI", "TRMM_MX", "SLICE_A", "SLICE_X", "RESID_SL",
    "SLICE_W", "SLICE_U", "TRMM_SL", "TRTRI_COL")}


def task_spans(records, ntasks):
    """Per task: first item's start and last item's end (ns)."""
    st = records["t_start_ns"].astype(np.int64)
    en = records["t_end_ns"].astype(np.int64)
    ts = np.full(ntasks, np.iinfo(np.int64).max, dtype=np.int64)
    te = np.zeros(ntasks, dtype=np.int64)
    np.minimum.at(ts, records["task"], st)
    np.maximum.at(te, records["task"], en)
    return ts, te


def summary(records, ntasks, edges, nctas):
    """records: Context.trace_read() of one launch; edges: (pred, succ)
    pairs of that launch (Context.dag_edges() before the wait), each from an
    earlier to a later submission; nctas: the launch's grid.  Returns the
    makespan, the CTA busy fraction (item time over CTAs x makespan), the
    per-kind share of the CTA time, the critical path (its length, share of
    the makespan, task count, time per kind along it, and how long its tasks
    waited after their predecessor on it ended), and the number of edges
    whose successor started before its predecessor ended (0 for a legal
    run)."""
    ed = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    st = records["t_start_ns"].astype(np.int64)
    en = records["t_end_ns"].astype(np.int64)
    makespan = int(en.max()) - int(st.min())
    dur = en - st
    kinds = {}
    for k in np.unique(records["kind"]):
        m = records["kind"] == k
        kinds[KIND_NAMES.get(int(k), str(int(k)))] = {"items": int(m.sum()),
                                                      "cta_time_share": float(dur[m].sum() / dur.sum()),
                                                      "mean_item_us": float(dur[m].mean() / 1e3)}
    ts, te = task_spans(records, ntasks)
    span = te - ts
    # submission order is a topological order: one pass in task order
    order = np.argsort(ed[:, 1], kind="stable")
    preds, succ_of = ed[order, 0], ed[order, 1]
    first = np.searchsorted(succ_of, np.arange(ntasks + 1))
    cp = span.astype(np.float64)
    via = np.full(ntasks, -1, dtype=np.int64)      # predecessor on the longest chain
    for v in range(ntasks):
        a, z = first[v], first[v + 1]
        if z > a:
            j = a + int(np.argmax(cp[preds[a:z]]))
            cp[v] += cp[preds[j]]
            via[v] = preds[j]
    # the critical path itself: its tasks' spans per kind, and the time the
    # path's tasks waited after their chain predecessor ended (queueing)
    task_kind = np.full(ntasks, -1, dtype=np.int64)
    task_kind[records["task"]] = records["kind"]
    v = int(np.argmax(cp))
    path_kinds, waits, ntask_path = {}, 0, 0
    while v >= 0:
        name = KIND_NAMES.get(int(task_kind[v]), str(int(task_kind[v])))
        path_kinds[name] = path_kinds.get(name, 0.0) + float(span[v]) / 1e6
        if via[v] >= 0:
            waits += max(0, int(ts[v]) - int(te[via[v]]))
        ntask_path += 1
        v = int(via[v])
    return {"makespan_ms": makespan / 1e6, "cta_busy_frac": float(dur.sum()) / (nctas * makespan),
            "critical_path_ms": float(cp.max()) / 1e6, "critical_path_share": float(cp.max()) / makespan,
            "critical_path_tasks": ntask_path, "critical_path_ms_by_kind": path_kinds,
            "critical_path_wait_ms": waits / 1e6,
            "edges_violated": int(np.sum(te[ed[:, 0]] > ts[ed[:, 1]])) if len(ed) else 0, "kinds": kinds}
