"""Comparison helpers of the GPU parity tests.

Each comparison against the oracle checks two measures on the same arrays:

* the aggregate relative L2 error, ||got - ref|| / ||ref||, against the
  tolerance of the workload (FP32 path 1e-5 per block, BF16 path 2e-2 per
  block, op-level tolerances as each test states);
* a per-token bound: for every token (the last axis holds its channels), the
  largest absolute error over its channels divided by that token's reference
  RMS must stay within TOKEN_FACTOR x the same tolerance. A fault confined to
  a few tokens (the wrapping longitude tiles, the pole rows, a ragged tail
  tile) adds only about sqrt(fraction of tokens) to the aggregate norm and can
  pass the first test; it cannot pass the second.
"""
import numpy as np

TOKEN_FACTOR = 8.0


def rel_l2(got, ref) -> float:
    got = np.asarray(got, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def token_err(got, ref, channels: int) -> float:
    """max over tokens of max_c |got - ref| / RMS_c(ref) (tokens = rows of `channels` values)."""
    g = np.asarray(got, np.float64).reshape(-1, channels)
    r = np.asarray(ref, np.float64).reshape(-1, channels)
    rms = np.sqrt(np.mean(r * r, axis=1))
    return float(np.max(np.max(np.abs(g - r), axis=1) / np.maximum(rms, 1e-300)))


def assert_close(got, ref, tol: float, channels: int, what=""):
    """Both measures within bounds; returns (rel-L2, worst token error)."""
    err = rel_l2(got, ref)
    tok = token_err(got, ref, channels)
    assert np.isfinite(err) and err <= tol, (what, "rel-L2", err, tol)
    assert np.isfinite(tok) and tok <= TOKEN_FACTOR * tol, (what, "worst token", tok, TOKEN_FACTOR * tol)
    return err, tok


# ------------------------------------------------------------------------
# The oracle's attention on a large grid, split over worker processes.
# Workers are started with the "spawn" method (never forked from a process
# that has used the GPU). The bf16-valued qkv sits in one shared-memory block;
# each worker evaluates oracle.neighborhood_attention for a range of queries.

def _na_worker(args):
    import os
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    from multiprocessing import shared_memory

    from oracle import wm_oracle as orc
    name, shape, C, heads, lo, hi, nbr = args
    shm = shared_memory.SharedMemory(name=name)
    try:
        qkv = np.ndarray(shape, dtype=np.float32, buffer=shm.buf)
        o = orc.neighborhood_attention(qkv[:, lo:hi, :C], qkv[..., C:2 * C], qkv[..., 2 * C:], heads, nbr,
                                       chunk=128)
        return lo, o.astype(np.float64)
    finally:
        shm.close()


def na_oracle_parallel(qkv, C, heads, nbr, workers=12):
    """oracle.neighborhood_attention(q, k, v, heads, nbr) for qkv [B, N, 3C]
    (float32 holding bf16-representable values), all N queries, in `workers`
    spawned processes. Returns [B, N, C] float64."""
    import multiprocessing as mp
    from multiprocessing import shared_memory

    qkv = np.ascontiguousarray(qkv, dtype=np.float32)
    B, N, _ = qkv.shape
    shm = shared_memory.SharedMemory(create=True, size=qkv.nbytes)
    try:
        view = np.ndarray(qkv.shape, dtype=np.float32, buffer=shm.buf)
        view[...] = qkv
        bounds = np.linspace(0, N, workers + 1).astype(int)
        jobs = [(shm.name, qkv.shape, C, heads, int(lo), int(hi), nbr[lo:hi])
                for lo, hi in zip(bounds[:-1], bounds[1:]) if hi > lo]
        out = np.empty((B, N, C), dtype=np.float64)
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            for lo, o in pool.imap_unordered(_na_worker, jobs):
                out[:, lo:lo + o.shape[1]] = o
        return out
    finally:
        shm.close()
        shm.unlink()
