"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module holds no arithmetic of the factorisation method: it only builds
input matrices and initial factors with numpy's own generators, so the
oracle (``oracle/``) and the GPU library's tests and benchmark can be fed the
same bytes.  The random sketches the method draws at each iteration are NOT
made here: each side implements the Philox field itself.

Input recipes (stand-ins for the paper's datasets of Table 1, which are not
available offline):

  planted_dense      M = U0 V0^T + E,  U0, V0 ~ Uniform[0,1) with a given
                     fraction of entries zeroed, E_ij = |N(0, noise^2)|;
                     generated in row chunks of ``CHUNK`` rows, each chunk
                     from its own seeded stream, so any rows can be rebuilt
                     alone.  (dense image/video matrices BOATS/FACE/MNIST)
  sparse_text        CSR m documents x n terms; per-document length
                     round(LogNormal(ln(mean) - s^2/2, s)) clipped to [1, n];
                     term ids Zipf(a) on {1..n} (draws above n redrawn),
                     duplicates within a document merged; values log(1 + c)
                     with c ~ Poisson(1) conditioned on c >= 1.  (RCV1-like
                     text, Table 1)
  batch_specs        shapes of uneven planted instances: m ~ U{128..4096},
                     n ~ U{64..2048}, k in {8,16,32}, d = max(4k, n//8),
                     d' = max(4k, m//8).
"""
import concurrent.futures as _cf
import os

import numpy as np

CHUNK = 4096


def _chunk_rng(seed, tag, chunk):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(tag), int(chunk)])))


def planted_factors(m, n, k, seed, zero_frac=0.0):
    """U0 (m x k), V0 (n x k) ~ Uniform[0,1) (float32) with ``zero_frac`` zeroed."""
    g = _chunk_rng(seed, 1, 0)
    U0 = g.random((m, k), dtype=np.float32)
    V0 = g.random((n, k), dtype=np.float32)
    if zero_frac > 0:
        U0[g.random((m, k)) < zero_frac] = 0.0
        V0[g.random((n, k)) < zero_frac] = 0.0
    return U0, V0


def _planted_rows(U0, V0, seed, noise, r0, r1):
    g = _chunk_rng(seed, 2, r0 // CHUNK)
    n = V0.shape[0]
    E = g.standard_normal((r1 - r0, n), dtype=np.float32)
    np.abs(E, out=E)
    E *= np.float32(noise)
    E += U0[r0:r1] @ V0.T
    return E


def planted_dense(m, n, k, seed, zero_frac=0.0, noise=0.01, threads=None):
    """M (m x n float32, row-major), U0, V0 as described in the module header."""
    U0, V0 = planted_factors(m, n, k, seed, zero_frac)
    M = np.empty((m, n), dtype=np.float32)
    starts = list(range(0, m, CHUNK))

    def work(r0):
        r1 = min(m, r0 + CHUNK)
        M[r0:r1] = _planted_rows(U0, V0, seed, noise, r0, r1)

    threads = threads or min(32, os.cpu_count() or 1)
    if len(starts) == 1:
        work(0)
    else:
        with _cf.ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, starts))
    return M, U0, V0


def planted_dense_rows(m, n, k, seed, rows, zero_frac=0.0, noise=0.01):
    """The given rows of planted_dense(m, n, k, seed, ...) without building all of M."""
    U0, V0 = planted_factors(m, n, k, seed, zero_frac)
    rows = np.asarray(rows)
    out = np.empty((len(rows), n), dtype=np.float32)
    cache = {}
    for idx, i in enumerate(rows):
        c = int(i) // CHUNK
        if c not in cache:
            r0 = c * CHUNK
            cache[c] = _planted_rows(U0, V0, seed, noise, r0, min(m, r0 + CHUNK))
        out[idx] = cache[c][int(i) - c * CHUNK]
    return out


def initial_factors(m, n, k, seed):
    """U, V ~ Uniform[0,1) float32, independent of the planted factors."""
    g = _chunk_rng(seed, 3, 0)
    return g.random((m, k), dtype=np.float32), g.random((n, k), dtype=np.float32)


def sparse_text(m, n, seed, mean_len=100.0, sigma=1.0, zipf_a=1.07):
    """CSR (rowptr int64[m+1], col int32[nnz], val float32[nnz]); rows sorted by column."""
    g = _chunk_rng(seed, 4, 0)
    mu = np.log(mean_len) - 0.5 * sigma * sigma
    L = np.rint(g.lognormal(mu, sigma, size=m)).astype(np.int64)
    np.clip(L, 1, n, out=L)
    total = int(L.sum())
    cols = g.zipf(zipf_a, size=total)
    bad = cols > n
    while bad.any():
        cols[bad] = g.zipf(zipf_a, size=int(bad.sum()))
        bad = cols > n
    cols -= 1
    rows = np.repeat(np.arange(m, dtype=np.int64), L)
    keys = rows * np.int64(n) + cols.astype(np.int64)
    del rows, cols
    keys = np.unique(keys)
    r = keys // n
    c = (keys - r * n).astype(np.int32)
    counts = np.bincount(r, minlength=m)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    cnt = g.poisson(1.0, size=len(c))
    zero = cnt == 0
    while zero.any():
        cnt[zero] = g.poisson(1.0, size=int(zero.sum()))
        zero = cnt == 0
    val = np.log1p(cnt.astype(np.float64)).astype(np.float32)
    return rowptr, c, val


def batch_specs(count, seed):
    """List of dicts (m, n, k, d, d_v, seed) for uneven planted instances."""
    g = _chunk_rng(seed, 5, 0)
    specs = []
    for i in range(count):
        m = int(g.integers(128, 4097))
        n = int(g.integers(64, 2049))
        k = int(g.choice([8, 16, 32]))
        specs.append(dict(m=m, n=n, k=k, d=max(4 * k, n // 8), d_v=max(4 * k, m // 8), seed=i))
    return specs


def planted_dense_torch(m, n, k, seed, zero_frac=0.0, noise=0.01, device="cuda"):
    """Same recipe as planted_dense, drawn with torch's generator on `device`
    (fast, for large throw-away training matrices; not bit-identical to the
    numpy recipe).  Returns M (m x n float32 tensor)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 17)
    U0 = torch.rand((m, k), generator=g, device=device)
    V0 = torch.rand((n, k), generator=g, device=device)
    if zero_frac > 0:
        U0[torch.rand((m, k), generator=g, device=device) < zero_frac] = 0.0
        V0[torch.rand((n, k), generator=g, device=device) < zero_frac] = 0.0
    M = torch.randn((m, n), generator=g, device=device).abs_().mul_(noise)
    M.addmm_(U0, V0.T)
    return M
