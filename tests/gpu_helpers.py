"""Helpers for the GPU parity tests: move arc lists to the device and count
through the C ABI (via the thin binding)."""
import numpy as np

import synth


def csr_arrays(n, src, dst):
    return synth.arcs_to_csr(n, np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32))


def gpu_count(counter, n, src, dst, k, stream=None):
    import torch
    rowptr, col = csr_arrays(n, src, dst)
    r = torch.from_numpy(rowptr).cuda()
    c = torch.from_numpy(col).cuda()
    out = counter.count(r, c, n, k, stream=stream)
    torch.cuda.synchronize()
    return out.cpu().numpy()
