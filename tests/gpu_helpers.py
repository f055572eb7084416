"""Helpers of the GPU tests: run the library on a workload and map its basis onto the
oracle's by state identity (parity, modes)."""
import numpy as np
import torch

from paper_2410_04204_gb300 import tgba


class GpuSector:
    def __init__(self, handle, s, max_qp):
        info = tgba.tgba_basis_info(handle, s, max_qp)
        self.h, self.s = handle, s
        self.n_ns, self.n_r = info["n_ns"], info["n_r"]
        self.E0 = info["E0"]
        self.nqp = info["nqp"]
        self.keys = [(int(p), tuple(int(v) for v in row[:q]))
                     for p, row, q in zip(info["parity"], info["modes"], info["nqp"])]

    def x(self):
        out = torch.empty(self.n_ns * self.n_r, dtype=torch.complex128, device="cuda")
        if out.numel():
            tgba.tgba_x_export(self.h, self.s, out)
        return out.cpu().numpy().reshape(self.n_ns, self.n_r)

    def perm_to(self, ns, r):
        """Index arrays pa, pb with X_gpu[i, j] <-> X_oracle[pa[i], pb[j]]."""
        key = {(0, s.modes): i for i, s in enumerate(ns)}
        key.update({(1, s.modes): i for i, s in enumerate(r)})
        pa = np.array([key[k] for k in self.keys[:self.n_ns]], dtype=np.int64)
        pb = np.array([key[k] for k in self.keys[self.n_ns:]], dtype=np.int64)
        return pa, pb


def x_close(xg, xo, rel=1e-10):
    """|dX| <= rel (|X| + 1e-3 max|X|): elementwise relative, with a floor at the block scale
    for entries that are small only through cancellation."""
    scale = np.abs(xo).max() if xo.size else 1.0
    err = np.abs(xg - xo)
    return bool(np.all(err <= rel * (np.abs(xo) + 1e-3 * scale))), float((err / (np.abs(xo) + 1e-3 * scale)).max() if xo.size else 0.0)
