"""Small helpers for the GPU tests: numpy <-> CUDA tensors of 32-bit words."""
import numpy as np


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.uint32))).cuda()


def dev64(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.int64))).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


def assert_equal(got, want, what=""):
    got = np.asarray(got, dtype=np.uint32)
    want = np.asarray(want, dtype=np.uint32)
    assert got.shape == want.shape, f"{what}: shape {got.shape} vs {want.shape}"
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (f"{what}: {bad.size} of {got.size} words differ; first at {bad[:5]}: "
                           f"got {got[bad[:5]]} want {want[bad[:5]]}")
