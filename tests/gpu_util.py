"""Helpers for the GPU tests: numpy uint64 limbs <-> torch CUDA int64 tensors."""
import numpy as np


def dev(arr, device="cuda"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint64).view(np.int64)).to(device)


def host(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64).copy()


def gpu_hash(binding, blk_x, blk_a, blk_b, n, m, stream=None):
    import torch

    if stream is None:
        out = binding.hash(dev(blk_x), dev(blk_a), dev(blk_b), n, m)
    else:
        with torch.cuda.stream(stream):  # operands made and read on the hashing stream
            out = binding.hash(dev(blk_x), dev(blk_a), dev(blk_b), n, m, stream=stream)
    torch.cuda.synchronize()
    return host(out)
