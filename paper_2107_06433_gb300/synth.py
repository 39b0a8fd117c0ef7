"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on a 100,000 x 300 subset of fastText crawl embeddings and
the first 5,000 DBpedia training documents (Section III-B2).  Neither dataset is
available, so every input here is synthetic:

* embeddings: i.i.d. N(0, 1) rows, L2-normalised, float32;
* document word ids: truncated Zipf(s) over ranks 1..V, id = rank - 1, so id 0
  is the most frequent word, as in a frequency-sorted embedding file; the ids of
  one document are distinct (duplicates are re-drawn);
* counts: uniform integers 1..count_max, normalised so every document sums to 1;
* queries: distinct Zipf ids with uniform weights.

This module is shared by the CUDA path's tests and bench and by the oracle's
tests.  It holds none of the method's arithmetic: only random draws, sorting and
the CSR bookkeeping of the paper's input format (c is a V x N CSR matrix whose
columns sum to one, Section III-B1).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 210706433


def streams(seed: int = SEED, n: int = 4) -> list[np.random.Generator]:
    """Independent generators: [embeddings, documents, queries, arrivals]."""
    return [np.random.Generator(np.random.PCG64(s))
            for s in np.random.SeedSequence(seed).spawn(n)]


def embeddings(rng: np.random.Generator, V: int, d: int) -> np.ndarray:
    """V x d float32, rows i.i.d. N(0,1) then scaled to unit L2 norm."""
    E = rng.standard_normal((V, d), dtype=np.float32)
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    return np.ascontiguousarray(E, dtype=np.float32)


def zipf_cdf(V: int, s: float = 1.1) -> np.ndarray:
    w = np.arange(1, V + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_ids(rng: np.random.Generator, cdf: np.ndarray, n: int) -> np.ndarray:
    """n ids in [0, V) drawn from the truncated Zipf law given by its cdf."""
    ids = np.searchsorted(cdf, rng.random(n), side="right")
    return np.minimum(ids, len(cdf) - 1).astype(np.int64)


def _unique_per_doc(rng, cdf, doc_ptr):
    """Draw doc_ptr[-1] ids, distinct within each document, sorted ascending."""
    N = len(doc_ptr) - 1
    lens = np.diff(doc_ptr)
    total = int(doc_ptr[-1])
    V = len(cdf)
    if np.any(lens > V):
        raise ValueError("a document is longer than the vocabulary")
    doc_of = np.repeat(np.arange(N, dtype=np.int64), lens)
    ids = zipf_ids(rng, cdf, total)
    todo = np.arange(N, dtype=np.int64)          # documents still to check
    while todo.size:
        pos = np.concatenate([np.arange(doc_ptr[j], doc_ptr[j + 1]) for j in todo]) \
            if todo.size < 4096 else None
        if pos is None:
            mask = np.zeros(N, dtype=bool)
            mask[todo] = True
            pos = np.nonzero(mask[doc_of])[0]
        key = doc_of[pos] * V + ids[pos]
        order = np.argsort(key, kind="stable")
        spos = pos[order]
        skey = key[order]
        dup = np.zeros(spos.size, dtype=bool)
        dup[1:] = skey[1:] == skey[:-1]
        # write the sorted ids back so each document is ascending
        ids[pos] = ids[spos]
        if not dup.any():
            break
        # positions (after the write-back) that hold a repeated id
        bad = pos[dup]
        ids[bad] = zipf_ids(rng, cdf, bad.size)
        todo = np.unique(doc_of[bad])
    return ids


@dataclasses.dataclass
class Corpus:
    """Target documents.  doc-major arrays plus the paper's V x N CSR form."""
    V: int
    N: int
    doc_ptr: np.ndarray      # int64 [N+1]
    word_ids: np.ndarray     # int32 [nnz], ascending within a document
    counts: np.ndarray       # int32 [nnz]
    vals: np.ndarray         # float32 [nnz], counts / document total

    @property
    def nnz(self) -> int:
        return int(self.doc_ptr[-1])

    def csr(self):
        """(row_ptr int64[V+1], doc_idx int32[nnz], val float32[nnz]): c as V x N CSR."""
        doc_of = np.repeat(np.arange(self.N, dtype=np.int64), np.diff(self.doc_ptr))
        order = np.lexsort((doc_of, self.word_ids))
        row_cnt = np.bincount(self.word_ids, minlength=self.V)
        row_ptr = np.zeros(self.V + 1, dtype=np.int64)
        np.cumsum(row_cnt, out=row_ptr[1:])
        return (row_ptr, doc_of[order].astype(np.int32),
                np.ascontiguousarray(self.vals[order], dtype=np.float32))


def corpus(rng: np.random.Generator, V: int, N: int, lens: np.ndarray,
           count_max: int, s: float = 1.1) -> Corpus:
    lens = np.asarray(lens, dtype=np.int64)
    assert lens.shape == (N,) and np.all(lens >= 1)
    doc_ptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(lens, out=doc_ptr[1:])
    ids = _unique_per_doc(rng, zipf_cdf(V, s), doc_ptr)
    counts = rng.integers(1, count_max + 1, size=ids.size, dtype=np.int64)
    tot = np.add.reduceat(counts, doc_ptr[:-1]) if N else np.zeros(0, np.int64)
    vals = (counts / np.repeat(tot, lens)).astype(np.float32)
    return Corpus(V, N, doc_ptr, ids.astype(np.int32), counts.astype(np.int32), vals)


def uniform_lens(rng, N, lo, hi):
    return rng.integers(lo, hi + 1, size=N, dtype=np.int64)


def lognormal_lens(rng, N, mean=60.0, sigma=0.6, lo=10, hi=300):
    mu = math.log(mean) - sigma * sigma / 2
    x = np.rint(rng.lognormal(mu, sigma, size=N))
    return np.clip(x, lo, hi).astype(np.int64)


def query(rng: np.random.Generator, V: int, v_r: int, s: float = 1.1):
    """v_r distinct Zipf ids (int32) and uniform weights (float32)."""
    cdf = zipf_cdf(V, s)
    got: list[int] = []
    seen = set()
    while len(got) < v_r:
        for w in zipf_ids(rng, cdf, 2 * v_r):
            w = int(w)
            if w not in seen:
                seen.add(w)
                got.append(w)
                if len(got) == v_r:
                    break
    return np.array(got, dtype=np.int32), np.ones(v_r, dtype=np.float32)


# ---------------------------------------------------------------------------
# Workload recipes.  Sizes follow the paper's dataset statistics (Section
# III-B2: V = 100,000, embedding size 300, 5,000 targets, query of 19 words)
# and larger single-GPU shapes of the same structure.

@dataclasses.dataclass
class Workload:
    name: str
    V: int
    d: int
    N: int
    v_r: int
    lam: float
    max_iter: int
    len_kind: str            # "uniform" | "lognormal"
    len_lo: int
    len_hi: int
    count_max: int
    len_mean: float = 60.0


WORKLOADS = {
    # small correctness case: dense oracle finishes in well under a second
    "tiny": Workload("tiny", V=2_000, d=64, N=200, v_r=8, lam=1.0, max_iter=15,
                     len_kind="uniform", len_lo=5, len_hi=30, count_max=5),
    # paper-shaped single query (Section III-B2 statistics)
    "paper": Workload("paper", V=100_000, d=300, N=5_000, v_r=19, lam=1.0, max_iter=15,
                      len_kind="lognormal", len_lo=10, len_hi=300, count_max=10),
    # the paper's own nnz (173,087 over 5,000 docs, mean 34.6 words)
    "paper_short": Workload("paper_short", V=100_000, d=300, N=5_000, v_r=19, lam=1.0,
                            max_iter=15, len_kind="lognormal", len_lo=10, len_hi=300,
                            count_max=10, len_mean=34.6),
    # large corpus: 1M short documents, HBM-bound iteration
    "large": Workload("large", V=500_000, d=300, N=1_000_000, v_r=32, lam=1.0, max_iter=15,
                      len_kind="uniform", len_lo=5, len_hi=30, count_max=10),
    # batched multi-query corpus
    "batch": Workload("batch", V=100_000, d=300, N=100_000, v_r=32, lam=1.0, max_iter=15,
                      len_kind="uniform", len_lo=10, len_hi=200, count_max=10),
}


def make(w: Workload | str, seed: int = SEED, N: int | None = None):
    """(E, corpus, (query ids, weights)) for a workload; N overrides the doc count."""
    if isinstance(w, str):
        w = WORKLOADS[w]
    N = w.N if N is None else N
    r_emb, r_doc, r_q, _ = streams(seed)
    E = embeddings(r_emb, w.V, w.d)
    if w.len_kind == "uniform":
        lens = uniform_lens(r_doc, N, w.len_lo, w.len_hi)
    else:
        lens = lognormal_lens(r_doc, N, w.len_mean, 0.6, w.len_lo, w.len_hi)
    C = corpus(r_doc, w.V, N, lens, w.count_max)
    q = query(r_q, w.V, w.v_r)
    return E, C, q


def batch_queries(V: int, n: int, vr_lo: int, vr_hi: int, seed: int = SEED):
    """n queries with v_r uniform in [vr_lo, vr_hi]."""
    rng = streams(seed)[2]
    rng = np.random.Generator(np.random.PCG64(rng.integers(1 << 62)))
    out = []
    for _ in range(n):
        vr = int(rng.integers(vr_lo, vr_hi + 1))
        out.append(query(rng, V, vr))
    return out


def poisson_arrivals(rate_qps: float, n: int, seed: int = SEED) -> np.ndarray:
    """Arrival times in seconds of n requests of a Poisson process."""
    rng = streams(seed)[3]
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=n))
