"""Helpers for the GPU tests: device buffers via torch, calls via the C ABI."""
import numpy as np
import torch

from paper_2605_30294_gb300 import rafi


def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def stream():
    return torch.cuda.current_stream(dev())


def to_dev(a: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(a).to(dev())


def zeros_u8(n, width):
    return torch.zeros((max(n, 1), width), dtype=torch.uint8, device=dev())


def exchange_once(R, item_bytes, items, dest, capacity=None, allow=(rafi.RF_ERR_OVERFLOW, rafi.RF_ERR_BAD_DEST)):
    """Push (items, dest) from device memory, exchange once, snapshot the incoming queue."""
    n = len(dest)
    cap = capacity or max(n, 1)
    s = stream()
    with rafi.Context(R, item_bytes, cap) as ctx:
        di = to_dev(items.reshape(n, item_bytes) if n else np.zeros((1, item_bytes), np.uint8))
        dd = to_dev(dest if n else np.zeros(1, np.int32))
        rafi.rf_push(ctx.handle, di, dd, n, False, s)
        st, na = rafi.rf_exchange(ctx.handle, s, allow=allow)
        out = zeros_u8(cap, item_bytes)
        off = torch.zeros(R + 1, dtype=torch.int32, device=dev())
        rafi.rf_snapshot(ctx.handle, out, off, s, allow=allow)
        stats = rafi.rf_stats(ctx.handle, allow=allow)
        torch.cuda.synchronize()
        return st, na, out[:na].cpu().numpy(), off.cpu().numpy().astype(np.uint64), stats


def canonical_rows(a: np.ndarray) -> np.ndarray:
    """Rows sorted lexicographically (canonical order of an unordered queue)."""
    if len(a) == 0:
        return a
    return a[np.lexsort(a.T[::-1])]
