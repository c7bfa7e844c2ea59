"""Raw CNF batches for the GPU tests: pack [(nvars, clauses)] into the C
ABI's CSR layout, solve through scuba_solve_batch_ex, check models."""
import numpy as np
import torch


def pack(cnfs):
    """[(nvars, list of clauses)] -> host CSR arrays."""
    icb, cb, lits, nv, vb = [0], [0], [], [], [0]
    for n, cls in cnfs:
        for c in cls:
            lits.extend(c)
            cb.append(len(lits))
        icb.append(len(cb) - 1)
        nv.append(n)
        vb.append(vb[-1] + n)
    return (np.array(icb, np.int64), np.array(cb, np.int64), np.array(lits or [0], np.int32),
            np.array(nv or [0], np.int32), np.array(vb, np.int64), len(lits))


def solve_raw(api, cnfs, **opts):
    from paper_2601_21552_gb300 import binding as B
    icb, cb, lits, nv, vb, L = pack(cnfs)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(a).to(dev)
    d_icb, d_cb, d_lits, d_nv, d_vb = t(icb), t(cb), t(lits), t(nv), t(vb)
    n = len(cnfs)
    b = B.make_batch(n, int(max(nv.max(), 0)) if n else 0, len(cb) - 1, L, int(vb[-1]),
                     d_icb.data_ptr(), d_cb.data_ptr(), d_lits.data_ptr(), d_nv.data_ptr(),
                     d_vb.data_ptr())
    verdict = torch.full((max(n, 1),), 9, dtype=torch.uint8, device=dev)
    model = torch.zeros(max(int(vb[-1]), 1), dtype=torch.uint8, device=dev)
    stats = torch.zeros((max(n, 1), B.SCUBA_NSTATS), dtype=torch.int64, device=dev)
    o = api.options(stats=stats, time_budget_ms=opts.pop("time_budget_ms", 60000), **opts)
    B.scuba_solve_batch_ex(b, verdict.data_ptr(), model.data_ptr(),
                           torch.cuda.current_stream().cuda_stream, o)
    st = B.scuba_sync_status(torch.cuda.current_stream().cuda_stream)
    return st, verdict.cpu().numpy()[:n], model.cpu().numpy(), vb, stats.cpu().numpy()[:n]


def model_ok(cls, model, base):
    return all(any((model[base + abs(l) - 1] == 1) == (l > 0) for l in c) for c in cls)
