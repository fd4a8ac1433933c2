"""Shared helpers of the GPU tests: device blocks through torch, comparison
against the oracle."""
import numpy as np

import oracle


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def to_dev(a, dtype="c128"):
    torch = torch_cuda()
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128 if dtype == "c128" else np.complex64))
    return t.cuda()


def empty_dev(shape, dtype="c128"):
    torch = torch_cuda()
    return torch.empty(shape, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device="cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def osys(w):
    return oracle.System(**{k: v for k, v in w.items() if k != "name"})


def sampled_rows_reference(w, x_dev, rows):
    """(H x)[mu] for sampled rows mu, by the oracle from columns of H and
    Hermiticity, reading only the needed entries of the device block x."""
    torch = torch_cuda()
    s = osys(w)
    out = []
    for mu in rows:
        r, v = oracle.h_column(s, int(mu))
        xr = x_dev[torch.from_numpy(r).cuda()].cpu().numpy().astype(np.complex128)
        out.append((np.conj(v)[:, None] * xr).sum(axis=0))
    return np.array(out)
