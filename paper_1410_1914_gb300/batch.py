"""Many structures in one persistent launch, with a cached autotuner.

``Batch`` groups ``Solver`` objects (each with its structure loaded) and
drives the batch entry points of the C ABI.  ``Batch.autotune`` times the
tile shape, work-item z length and L2 prefetch distance on the GPU and caches
the result in a JSON file keyed by storage mode and the members' box sizes,
so the next batch of the same shape skips the trials.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import _lib as L

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "cl_lbm_autotune.json")


class Batch:
    def __init__(self, solvers, z_chunk: int = 0):
        self.solvers = list(solvers)
        self.b = L.cl_batch_create([s.h for s in self.solvers], z_chunk)

    def close(self):
        if getattr(self, "b", None):
            L.cl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        self.close()

    def step(self, n: int):
        L.cl_batch_step(self.b, n)

    def solve(self, max_steps: int):
        status, infos, nconv = L.cl_batch_solve(self.b, len(self.solvers), max_steps)
        return L.status_str(status), infos, nconv

    def configure(self, z_chunk: int, prefetch: int, tile_rows: int):
        """tile_rows: 1, 2, 4 rows per warp for every member, 0: each member's own shape."""
        L.cl_batch_configure(self.b, z_chunk, prefetch, tile_rows)

    def info(self):
        return L.cl_batch_info(self.b)

    def signature(self) -> str:
        sizes = sorted(tuple(s.shape) for s in self.solvers)
        storage = int(self.solvers[0].params.storage)
        return hashlib.sha256(json.dumps([storage, sizes]).encode()).hexdigest()[:16]

    def autotune(self, steps_per_trial: int = 20, cache: str | None = DEFAULT_CACHE):
        """(z_chunk, prefetch, tile_rows, ms_per_step, from_cache)."""
        key = self.signature()
        table = {}
        if cache and os.path.exists(cache):
            try:
                with open(cache) as fh:
                    table = json.load(fh)
            except (OSError, ValueError):
                table = {}
        if key in table and len(table[key]) == 4:
            zc, pf, tr, ms = table[key]
            self.configure(zc, pf, tr)
            return zc, pf, tr, ms, True
        zc, pf, tr, ms = L.cl_batch_autotune(self.b, steps_per_trial)
        if cache:
            table[key] = [zc, pf, tr, ms]
            os.makedirs(os.path.dirname(cache), exist_ok=True)
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh)
            os.replace(tmp, cache)
        return zc, pf, tr, ms, False
