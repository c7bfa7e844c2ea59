"""Torch-facing convenience layer over the C ABI.

torch provides device memory and streams only; encoding, solving and
verification all happen in libscuba. The functions here marshal tensors into
the ``scuba_cnf_batch`` / ``scuba_options`` structs and call the ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import binding as B


class DeviceBatch:
    """The CSR of an encoded batch resident on a CUDA device (torch tensors)."""

    def __init__(self, enc: B.Encoded, device: str | torch.device = "cuda", pin: bool = True):
        self.enc = enc
        self.n = enc.n
        self.max_vars = enc.max_vars
        self.total_clauses = enc.total_clauses
        self.total_lits = enc.total_lits
        self.total_vars = enc.total_vars
        dev = torch.device(device)

        def up(a: np.ndarray) -> torch.Tensor:
            t = torch.from_numpy(np.ascontiguousarray(a))
            if pin:
                t = t.pin_memory()
            return t.to(dev, non_blocking=True)

        self.icb = up(enc.inst_clause_begin)
        self.cb = up(enc.clause_begin)
        self.lits = up(enc.lits if len(enc.lits) else np.zeros(1, np.int32))
        self.nv = up(enc.inst_num_vars if self.n else np.zeros(1, np.int32))
        self.vb = up(enc.inst_var_begin)
        self.h2d_bytes = sum(int(x.nbytes) for x in (enc.inst_clause_begin, enc.clause_begin,
                                                       enc.lits, enc.inst_num_vars,
                                                       enc.inst_var_begin))
        # input bits per instance (the encoder numbers them first): a feature
        # of the branching network
        iib, widths, _ = enc.inputs()
        csum = np.concatenate([[0], np.cumsum(widths, dtype=np.int64)])
        ninp = (csum[iib[1:]] - csum[iib[:-1]]).astype(np.int32) if self.n else np.zeros(1, np.int32)
        self.num_inputs = up(ninp if self.n else np.zeros(1, np.int32))

    @classmethod
    def from_csr(cls, icb, cb, lits, nv, vb, num_inputs=None, device="cuda", pin=True):
        """A device batch from host CSR arrays (inst_clause_begin, clause_begin,
        lits, inst_num_vars, inst_var_begin), e.g. DIMACS-style CNFs."""
        class _Enc:
            pass
        e = _Enc()
        e.n = len(nv)
        e.inst_clause_begin = np.ascontiguousarray(icb, np.int64)
        e.clause_begin = np.ascontiguousarray(cb, np.int64)
        e.lits = np.ascontiguousarray(lits, np.int32)
        e.inst_num_vars = np.ascontiguousarray(nv, np.int32)
        e.inst_var_begin = np.ascontiguousarray(vb, np.int64)
        e.total_clauses = len(cb) - 1
        e.total_lits = int(cb[-1]) if len(cb) else 0
        e.total_vars = int(vb[-1]) if len(vb) else 0
        e.max_vars = int(nv.max()) if len(nv) else 0
        ni = np.zeros(max(e.n, 1), np.int32) if num_inputs is None else np.asarray(num_inputs, np.int32)
        e.inputs = lambda: (np.zeros(e.n + 1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
        obj = cls(e, device, pin)
        obj.num_inputs = torch.from_numpy(ni).to(torch.device(device))
        return obj

    def lpt_order(self) -> torch.Tensor:
        """Largest instances first (longest-processing-time order by clause
        count), as a device int32 permutation for scuba_options.order."""
        if getattr(self, "_lpt", None) is None:
            nc = np.diff(self.enc.inst_clause_begin)
            perm = np.argsort(-nc, kind="stable").astype(np.int32)
            self._lpt = torch.from_numpy(perm).to(self.icb.device)
        return self._lpt

    def struct(self) -> B.scuba_cnf_batch:
        return B.make_batch(self.n, self.max_vars, self.total_clauses, self.total_lits,
                            self.total_vars, self.icb.data_ptr(), self.cb.data_ptr(),
                            self.lits.data_ptr(), self.nv.data_ptr(), self.vb.data_ptr())


class Trace:
    """Device buffers of a decision trace (scuba_trace), torch-owned."""

    def __init__(self, depth: int, max_nodes: int, max_rows: int, device="cuda"):
        dev = torch.device(device)
        z = lambda n, dt: torch.zeros(max(n, 1), dtype=dt, device=dev)
        self.depth, self.max_nodes, self.max_rows = depth, max_nodes, max_rows
        self.counts = z(2, torch.int64)
        self.node_inst = z(max_nodes, torch.int32)
        self.node_depth = z(max_nodes, torch.int32)
        self.node_row = z(max_nodes, torch.int64)
        self.node_nrows = z(max_nodes, torch.int32)
        self.node_closed = z(max_nodes, torch.int32)
        self.x = z(max_rows * 16, torch.int16)
        self.target = z(max_rows, torch.float32)
        self.var = z(max_rows, torch.int32)

    def struct(self) -> B.scuba_trace:
        t = B.scuba_trace()
        t.depth, t.max_nodes, t.max_rows = self.depth, self.max_nodes, self.max_rows
        for name in ("counts", "node_inst", "node_depth", "node_row", "node_nrows",
                     "node_closed", "x", "target", "var"):
            setattr(t, name, getattr(self, name).data_ptr())
        return t

    def used(self) -> tuple[int, int]:
        """(nodes, rows) actually recorded (capped at the capacities)."""
        c = self.counts.cpu().tolist()
        return min(c[0], self.max_nodes), min(c[1], self.max_rows)


SEARCH = {"dpll": B.SCUBA_SEARCH_DPLL, "cdcl": B.SCUBA_SEARCH_CDCL}


def options(heuristic: int = B.SCUBA_HEUR_ACTIVITY, decision_budget: int = 0,
            time_budget_ms: int = 0, split: bool = True, warps_per_block: int = 0,
            blocks_per_sm: int = 0, split_interval: int = 0, split_min: int = 0, trail_placement: int = 0, stats: torch.Tensor | None = None,
            order: torch.Tensor | None = None, mlp_weights: torch.Tensor | None = None,
            learned_depth: int = 0, abort_flag_ptr: int | None = None,
            events: tuple | None = None, finish_ns: torch.Tensor | None = None,
            profile: torch.Tensor | None = None, num_inputs: torch.Tensor | None = None,
            trace: "Trace | None" = None, search: str | int = "dpll",
            restart_unit: int = 0, learnt_words: int = 0,
            split_depth: int = 0, share_lbd: int = 0) -> B.scuba_options:
    o = B.scuba_options_init()
    o.heuristic = heuristic
    o.search = SEARCH[search] if isinstance(search, str) else int(search)
    o.restart_unit = restart_unit
    o.learnt_words = learnt_words
    o.split_depth = split_depth
    o.share_lbd = share_lbd
    o.decision_budget = decision_budget
    o.time_budget_ms = time_budget_ms
    o.split = 1 if split else 0
    o.warps_per_block = warps_per_block
    o.blocks_per_sm = blocks_per_sm
    o.split_interval = split_interval
    o.split_min = split_min
    o.trail_placement = trail_placement
    o.stats = stats.data_ptr() if stats is not None else None
    o.order = order.data_ptr() if order is not None else None
    o.mlp_weights = mlp_weights.data_ptr() if mlp_weights is not None else None
    o.learned_depth = learned_depth
    o.abort_flag = abort_flag_ptr
    o.inst_num_inputs = num_inputs.data_ptr() if num_inputs is not None else None
    if trace is not None:
        o._trace_keep = trace.struct()          # keep the struct alive with the options
        o.trace = ctypes.addressof(o._trace_keep)
    o.finish_ns = finish_ns.data_ptr() if finish_ns is not None else None
    o.profile = profile.data_ptr() if profile is not None else None
    if events is not None:
        o.search_event_begin = events[0].cuda_event
        o.search_event_end = events[1].cuda_event
    return o


def solve(db: DeviceBatch, want_model: bool = True, stats: bool = True,
          stream: torch.cuda.Stream | None = None, **opts):
    """Launch scuba_solve_batch_ex on `stream` (torch's current stream by
    default) and return (verdict u8[n], model u8[total_vars] | None,
    stats i64[n,3] | None) device tensors. Asynchronous: call
    ``status(stream)`` to wait and collect the device status."""
    dev = db.icb.device
    if opts.pop("tuned", False):
        from . import autotune
        tuned = autotune.load()
        if opts.get("search") == "cdcl":
            tuned.update(autotune.load(section="best_cdcl"))
        for k, v in tuned.items():
            opts.setdefault(k, v)
    if opts.get("order") == "lpt":
        opts["order"] = db.lpt_order()
    verdict = torch.empty(max(db.n, 1), dtype=torch.uint8, device=dev)
    model = torch.zeros(max(db.total_vars, 1), dtype=torch.uint8, device=dev) if want_model else None
    st = torch.zeros((max(db.n, 1), B.SCUBA_NSTATS), dtype=torch.int64, device=dev) if stats else None
    opts.setdefault("num_inputs", db.num_inputs)
    o = options(stats=st, **opts)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    B.scuba_solve_batch_ex(db.struct(), verdict.data_ptr(),
                           model.data_ptr() if model is not None else None,
                           s.cuda_stream, o)
    return verdict[:db.n], (model[:db.total_vars] if model is not None else None), \
        (st[:db.n] if st is not None else None)


def solve_units(db: DeviceBatch, unit_inst, asm_begin=None, asm_lits=None,
                want_model: bool = True, stream: torch.cuda.Stream | None = None, **opts):
    """Launch scuba_solve_units: unit u is instance unit_inst[u] of the batch
    under the DIMACS assumption literals asm_lits[asm_begin[u]:asm_begin[u+1]]
    (numpy or tensors). Returns (verdict u8[n_units], model u8 | None, model
    offset of each unit i64[n_units]) device tensors; asynchronous like
    solve()."""
    dev = db.icb.device
    if opts.pop("tuned", False):
        from . import autotune
        tuned = autotune.load()
        if opts.get("search") == "cdcl":
            tuned.update(autotune.load(section="best_cdcl"))
        for k, v in tuned.items():
            opts.setdefault(k, v)
    t = lambda a, dt: torch.as_tensor(np.asarray(a), dtype=dt).to(dev)
    host = lambda a: (a.cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a))
    ui_h = host(unit_inst).astype(np.int64).reshape(-1)
    n_units = len(ui_h)
    if asm_begin is not None:  # the offsets the kernels will follow into asm_lits
        ab_h = host(asm_begin).astype(np.int64).reshape(-1)
        n_lits = len(host(asm_lits).reshape(-1)) if asm_lits is not None else 0
        if len(ab_h) != n_units + 1 or ab_h[0] < 0 or (np.diff(ab_h) < 0).any() \
                or ab_h[-1] > n_lits:
            raise ValueError("asm_begin must hold n_units + 1 non-negative, non-decreasing "
                             "offsets into asm_lits")
        asm_begin = ab_h
        asm_lits = host(asm_lits) if asm_lits is not None else None
    ui = t(ui_h.astype(np.int32), torch.int32)
    ab = t(asm_begin, torch.int64) if asm_begin is not None else None
    al = t(asm_lits if asm_lits is not None and len(asm_lits) else [0], torch.int32) \
        if asm_begin is not None else None
    # model offsets on the host: an out-of-range instance index (the kernels
    # report it and leave the unit UNKNOWN) takes no model space
    nv_h = np.asarray(db.enc.inst_num_vars, dtype=np.int64)
    ok = (ui_h >= 0) & (ui_h < db.n)
    nvu = np.where(ok, nv_h[np.where(ok, ui_h, 0)] if db.n else 0, 0)
    mb_h = np.zeros(max(n_units, 1), np.int64)
    if n_units:
        mb_h[1:n_units] = np.cumsum(nvu)[:-1]
    mb = t(mb_h, torch.int64)
    total = int(nvu.sum()) if n_units else 0
    verdict = torch.empty(max(n_units, 1), dtype=torch.uint8, device=dev)
    model = torch.zeros(max(total, 1), dtype=torch.uint8, device=dev) if want_model else None
    opts.setdefault("num_inputs", db.num_inputs)
    o = options(**opts)
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    B.scuba_solve_units(db.struct(), n_units, ui.data_ptr(),
                        ab.data_ptr() if ab is not None else None,
                        al.data_ptr() if al is not None else None,
                        mb.data_ptr() if model is not None else None, verdict.data_ptr(),
                        model.data_ptr() if model is not None else None, s.cuda_stream, o)
    return verdict[:n_units], model, mb[:n_units]


def status(stream: torch.cuda.Stream | None = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return B.scuba_sync_status(s.cuda_stream)


def solve_queries(irs: list, device: str = "cuda", **opts):
    """Encode on the host, upload, solve, re-verify every SAT model on the
    host. Returns dict(verdict, stats, verified, enc)."""
    enc = B.scuba_encode_batch(irs)
    db = DeviceBatch(enc, device)
    v, m, st = solve(db, **opts)
    rc = status()
    vh = v.cpu().numpy()
    mh = m.cpu().numpy() if m is not None else np.zeros(1, np.uint8)
    fails, ok = B.scuba_verify_batch(enc, vh, mh)
    return dict(verdict=vh, stats=st.cpu().numpy() if st is not None else None,
                verified=ok, fails=fails, status=rc, enc=enc, model=mh)


class Mlp:
    """The branching network: FP32 master parameters, Adam moments and the
    packed BF16 weights the solver reads, all device tensors."""

    def __init__(self, seed: int = 1, device="cuda"):
        dev = torch.device(device)
        self.master = torch.zeros(B.SCUBA_MLP_NPARAM, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.weights = torch.zeros(B.SCUBA_MLP_WEIGHT_BYTES, dtype=torch.uint8, device=dev)
        s = torch.cuda.current_stream(dev).cuda_stream
        B._check(B._lib.scuba_mlp_init(self.master.data_ptr(), self.weights.data_ptr(),
                                       ctypes.c_uint64(seed), s), "scuba_mlp_init")

    def train(self, trace: Trace, epochs: int = 10, batch_nodes: int = 64, lr: float = 3e-3):
        """Adam over the recorded nodes; returns the mean loss per epoch."""
        nodes, _ = trace.used()
        loss = torch.zeros(2 * max(epochs, 1), dtype=torch.float32, device=self.master.device)
        t = trace.struct()
        s = torch.cuda.current_stream(self.master.device).cuda_stream
        B._check(B._lib.scuba_mlp_train(ctypes.byref(t), nodes, self.master.data_ptr(),
                                        self.m.data_ptr(), self.v.data_ptr(),
                                        self.weights.data_ptr(), epochs, batch_nodes,
                                        ctypes.c_float(lr), loss.data_ptr(), s),
                 "scuba_mlp_train")
        lh = loss.cpu().numpy().reshape(-1, 2)[:epochs]
        return (lh[:, 0] / np.maximum(lh[:, 1], 1)).tolist()


def record_trace(db: DeviceBatch, depth: int = 6, max_nodes: int = 1 << 16,
                 max_rows: int = 1 << 24, decision_budget: int = 0, time_budget_ms: int = 0):
    """Run the plain search in trace mode (one warp per instance) and return
    (Trace, verdict, stats)."""
    tr = Trace(depth, max_nodes, max_rows, db.icb.device)
    v, _, st = solve(db, want_model=False, trace=tr, decision_budget=decision_budget,
                     time_budget_ms=time_budget_ms, split=False)
    rc = status()
    if rc != 0:
        raise RuntimeError(f"trace solve failed with status {rc}")
    return tr, v, st
