"""Checkpointed envelope jobs: a long simulation envelope runs in chunks of realizations and can
resume after an interruption.

The simulation generator is counter-based (realization k of a job is a pure function of the
seed and k), so a chunk is recomputed exactly and the chunks' per-realization grids, stored
as they finish, make up the whole job bit for bit; the envelope is their element-wise min /
max.  Host logic only: every realization is computed by the library (``stk_run``).
"""
from __future__ import annotations

import os

import numpy as np

from . import _lib


def envelope_resumable(pattern, s, tt, n_sims, seed, path, chunk=16, max_chunks=None, **kw):
    """Observed grids plus the envelope over realizations 0..n_sims-1, computed `chunk`
    realizations at a time; finished chunks are saved to ``path`` (a directory) and skipped
    when the call is repeated.  ``max_chunks`` stops after that many new chunks (returns None
    when the job is not complete yet).  ``kw`` goes to ``stk_run`` (precision, edge mode,
    simulation method, ...).  Returns the dict of ``stk_run`` with ``K_sims`` / ``C_sims`` for
    all realizations."""
    s, tt = np.asarray(s, np.float64), np.asarray(tt, np.float64)
    os.makedirs(path, exist_ok=True)
    done_now = 0
    for first in range(0, n_sims, chunk):
        m = min(chunk, n_sims - first)
        f = os.path.join(path, f"sims_{first:08d}_{m:06d}.npz")
        if os.path.exists(f):
            continue
        if max_chunks is not None and done_now >= max_chunks:
            return None
        r = _lib.stk_run(pattern.h, s, tt, n_sims=m, seed=seed, first_sim=first, want_sims=True,
                         **kw)
        tmp = f + ".tmp.npz"
        np.savez(tmp, K=r["K_sims"], C=r["C_sims"])
        os.replace(tmp, f)
        done_now += 1
    obs = _lib.stk_run(pattern.h, s, tt, n_sims=0, seed=seed, **kw)
    Ks, Cs = [], []
    for first in range(0, n_sims, chunk):
        m = min(chunk, n_sims - first)
        z = np.load(os.path.join(path, f"sims_{first:08d}_{m:06d}.npz"))
        Ks.append(z["K"])
        Cs.append(z["C"])
    Ks, Cs = np.concatenate(Ks), np.concatenate(Cs)
    # the envelope (min / max over realizations) and its L (Eq. 4, with the sector factor of a
    # directional K) are computed by the library
    obs.update(K_sims=Ks, C_sims=Cs)
    obs.update(_lib.stk_envelope_merge(Ks, s, tt, n_sectors=kw.get("n_sectors", 0)))
    return obs
