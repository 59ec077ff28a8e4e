"""The FP64 oracle evaluated over many host cores, for parity checks at the full workload sizes.

Test infrastructure only.  Every number still comes from ``oracle.cpm_oracle`` as it stands: the
elastance rows and the site values of b are independent of one another (``assemble_A(rows=...)``,
``bvec(sites=...)``), so chunks of rows and of sites are handed to worker processes and the pieces
are stacked in order.  Nothing is reordered inside a chunk, so the result equals the one-process
call up to the thread count of the BLAS inside each matrix product.

The pool is started with the ``spawn`` method (a forked child of a process that already holds a
CUDA context can hang), with one BLAS thread per worker.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

from oracle import cpm_oracle as o

_THREAD_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _rows(args):
    el, rows = args
    return o.assemble_A(el, rows=rows)


def _sites(args):
    el, ely, sites = args
    return o.bvec(el, ely, sites=sites)


class OraclePool:
    """``with OraclePool() as p: A = p.assemble_A(el); bs = p.bvec(el, [ely, ...])``."""

    def __init__(self, procs: int | None = None):
        self.procs = procs or max(1, min(32, os.cpu_count() or 1))
        self.pool = None

    def __enter__(self):
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        os.environ.update({k: "1" for k in _THREAD_VARS})
        try:
            self.pool = mp.get_context("spawn").Pool(self.procs)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return self

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()

    def _chunks(self, n, per_proc=4):
        k = max(1, min(n, self.procs * per_proc))
        return [c for c in np.array_split(np.arange(n), k) if len(c)]

    def assemble_A(self, el) -> np.ndarray:
        # one chunk per worker: every chunk evaluates the phases of all sites once
        parts = self.pool.map(_rows, [(el, c) for c in self._chunks(el.n, per_proc=1)])
        return np.vstack(parts)

    def bvec(self, el, elyts) -> list[np.ndarray]:
        # every chunk evaluates its configuration's structure factor once: as few chunks per
        # configuration as keep all workers busy
        per = max(1, -(-self.procs // len(elyts)))
        chunks = [c for c in np.array_split(np.arange(el.n), min(el.n, per)) if len(c)]
        jobs = [(el, e, c) for e in elyts for c in chunks]
        parts = self.pool.map(_sites, jobs)
        out, k = [], 0
        for _ in elyts:
            out.append(np.concatenate(parts[k:k + len(chunks)]))
            k += len(chunks)
        return out


def oracle_S(el, pool: OraclePool | None = None, symm: bool = True):
    """(A, S) of the oracle; A assembled over the pool when one is given."""
    A = pool.assemble_A(el) if pool is not None else o.assemble_A(el)
    return A, o.capacitance_matrix(A, symm=symm)
