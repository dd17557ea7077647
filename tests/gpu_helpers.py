"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and lay
its outputs out like the oracle's."""
import numpy as np

import paper_2012_05695_b300 as ddm

TOL = 1e-4   # |D - D_oracle| / s_q, s_q = 2 var_t F(q, .)


def to_device(frames):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(frames))
    return t.cuda()


def gpu_structure_function(frames, n_bins=0, **kw):
    """D [H, W/2+1, N] (numpy float32) from the CUDA path; also the plan."""
    import torch
    N, H, W = frames.shape
    dtype = "u16" if frames.dtype == np.uint16 else "f32"
    plan = ddm.Plan(H, W, N, dtype=dtype, n_bins=n_bins, **kw)
    f = to_device(frames)
    D = torch.empty(plan.n_q * N, dtype=torch.float32, device="cuda")
    plan.structure_function(f, D)
    torch.cuda.synchronize()
    return D.cpu().numpy().reshape(H, W // 2 + 1, N), plan, D


def storage_to_plane(spec, H, W):
    """Spectrum storage [N, n_q] complex -> [N, H, W/2+1] in (ky, kx) order."""
    ky, kx = ddm.spectrum_index_map(H, W)
    out = np.zeros((spec.shape[0], H, W // 2 + 1), dtype=spec.dtype)
    out[:, ky, kx] = spec
    return out


def plane_to_storage(F, H, W):
    """[N, H, W/2+1] complex -> spectrum storage [N, n_q]."""
    ky, kx = ddm.spectrum_index_map(H, W)
    return np.ascontiguousarray(F[:, ky, kx])


def oracle_columns_of_device_stack(frames_dev, cols, chunk=128):
    """The oracle's spectrum F [N, H, len(cols)] (complex128) of a float32 stack that lives
    on the device: frames are copied to the host a chunk at a time (a 1024x1024x4096 stack
    is 17 GB) and transformed by the oracle's own DFT restricted to the columns ``cols``."""
    import oracle
    N = frames_dev.shape[0]
    parts = []
    for t0 in range(0, N, chunk):
        host = frames_dev[t0:t0 + chunk].cpu().numpy()
        parts.append(oracle.dft2(host, cols))
    return np.concatenate(parts, axis=0)
