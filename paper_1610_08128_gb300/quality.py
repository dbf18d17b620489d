"""What an ordering buys: bandwidth, profile and sparse matrix-vector product time of P A P^T.

The paper motivates RCM by the cost of sparse kernels on badly ordered matrices (Sec. I, Fig. 1:
conjugate-gradient time on a mesh matrix before and after the ordering). This module measures the
single-GPU counterpart: the bandwidth and profile of the pattern (Sec. II-A) and the time of
y = A x with cuSPARSE's CSR SpMV (through torch), in the original and in the RCM order. It runs
outside the ordering path; the permuted matrix is built with torch operations on the device.
"""
from __future__ import annotations

import statistics


def permute_csr(rowptr, colidx, perm):
    """P A P^T of a CSR pattern on the device: perm[k] = old vertex at new position k (int32 CUDA
    tensors). Returns (rowptr, colidx) of the permuted pattern, columns sorted within rows."""
    import torch

    n = perm.numel()
    dev = perm.device
    p = perm.long()
    pos = torch.empty(n, dtype=torch.long, device=dev)
    pos[p] = torch.arange(n, dtype=torch.long, device=dev)
    lens = (rowptr[1:] - rowptr[:-1]).long()
    new_lens = lens[p]
    new_rowptr = torch.zeros(n + 1, dtype=torch.long, device=dev)
    new_rowptr[1:] = torch.cumsum(new_lens, 0)
    nnz = int(new_rowptr[-1])
    row = torch.repeat_interleave(torch.arange(n, dtype=torch.long, device=dev), new_lens, output_size=nnz)
    src = rowptr[:-1].long()[p][row] + (torch.arange(nnz, dtype=torch.long, device=dev) - new_rowptr[row])
    cols = pos[colidx.long()[src]]
    order = torch.argsort(row * n + cols)
    return new_rowptr.to(torch.int32), cols[order].to(torch.int32)


def spmv_ms(rowptr, colidx, repeats: int = 20) -> float:
    """Median time of y = A x (fp32 values 1, fp32 x) with cuSPARSE's CSR SpMV, in ms."""
    import torch

    import warnings

    n = rowptr.numel() - 1
    vals = torch.ones(colidx.numel(), dtype=torch.float32, device=colidx.device)
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", UserWarning)  # torch labels its sparse CSR support "beta"
        a = torch.sparse_csr_tensor(rowptr, colidx, vals, size=(n, n))
    x = torch.rand(n, 1, dtype=torch.float32, device=colidx.device)
    y = a @ x  # warm-up (and cuSPARSE set-up)
    stream = torch.cuda.current_stream()
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        y = a @ x
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    del y
    return statistics.median(times)


def report(rowptr, colidx, perm, repeats: int = 20) -> dict:
    """Bandwidth, profile and SpMV time of the pattern in its original order and in `perm`'s."""
    import torch

    from . import rcm

    n = perm.numel()
    ident = torch.arange(n, dtype=torch.int32, device=perm.device)
    bw0, prof0 = rcm.bandwidth_profile(rowptr, colidx, ident)
    bw1, prof1 = rcm.bandwidth_profile(rowptr, colidx, perm)
    prp, pci = permute_csr(rowptr, colidx, perm)
    t0 = spmv_ms(rowptr, colidx, repeats)
    t1 = spmv_ms(prp, pci, repeats)
    return {"bandwidth_original": bw0, "profile_original": prof0, "bandwidth_rcm": bw1, "profile_rcm": prof1,
            "spmv_ms_original": t0, "spmv_ms_rcm": t1, "spmv_speedup": t0 / t1 if t1 > 0 else None}
