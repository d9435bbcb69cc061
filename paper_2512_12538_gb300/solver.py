"""Convenience wrapper: one handle, torch tensors in and out."""
from __future__ import annotations

from . import _lib


class Solver:
    """Owns one libhh handle (set-up done in the constructor).

    Parameters follow ``hh_params`` (include/hh.h); ``precision`` is "fp64" or "mixed";
    ``k_rows`` (layered media) is one wavenumber per grid row.
    """

    def __init__(self, dim=2, n=255, k=40.0, levels=2, overlap=2, rank=16, oversample=10, n_inner=1,
                 tol=1e-10, max_iter=200, precision="fp64", seed=0, stream=None, leaf_solver="eigen",
                 outer="oras", restart=40, flags=0, k_rows=None):
        self.params = _lib.make_params(dim, n, k, levels, overlap, rank, oversample, n_inner, tol, max_iter,
                                       precision, seed, leaf_solver, outer, restart, flags, k_rows)
        self.S = n + 2
        self.Sx = self.S if dim == 2 else 1
        self.dim = dim
        self.handle, self.footprint = _lib.hh_setup(self.params, stream)

    def close(self):
        if self.handle is not None:
            _lib.hh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, f, g, stream=None, allow_noconv=False):
        """f [S][Sx], g [4][S] (or [2]) complex128 CUDA tensors -> (u, stats dict)."""
        import torch
        u = torch.empty((self.S, self.Sx), dtype=torch.complex128, device=f.device)
        st = _lib.hh_solve(self.handle, f.contiguous(), g.contiguous(), u, stream, allow_noconv)
        return u, st.as_dict()
