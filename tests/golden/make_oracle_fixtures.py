"""Writes stored oracle results for workloads too large to re-run in the GPU tests.

Calls only the oracle (and the seeded generators that feed it).  Usage:
    python tests/golden/make_oracle_fixtures.py rmat20 [--truss] [--ks 3,4,6,8]
    python tests/golden/make_oracle_fixtures.py batch10k_sample | serve_pool
writes tests/golden/<name>_oracle.txt.  Hashes are SHA-256 of the little-endian
int32 arrays in canonical edge order.  While it runs, the lines found so far
are kept in <name>_oracle.txt.partial (a scale-24 run takes hours), with the
time each step finished; the finished file replaces it at the end.
"""
import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import graphgen  # noqa: E402
import oracle  # noqa: E402


def sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype="<i4").tobytes()).hexdigest()


def batch_sample(n, count=200, bins=10, seed=7):
    """A seeded sample of a batch's graphs covering every size class: the
    graphs are split into `bins` log-spaced classes of n and the same number
    is drawn from each (all of a class that has fewer)."""
    rng = np.random.default_rng(seed)
    edges = np.exp(np.linspace(np.log(n.min()), np.log(n.max() + 1), bins + 1))
    cls = np.clip(np.searchsorted(edges, n, side="right") - 1, 0, bins - 1)
    pick = []
    for c in range(bins):
        idx = np.flatnonzero(cls == c)
        pick.extend(rng.choice(idx, min(len(idx), count // bins), replace=False).tolist())
    return sorted(pick)


def many_graphs(name):
    """Per-graph oracle results for the batch (a sample) and the serve pool
    (every graph): T and k-truss sizes."""
    lines = [f"# oracle results for {name}",
             "# written by tests/golden/make_oracle_fixtures.py (oracle only)"]
    t0 = time.time()
    if name == "batch10k_sample":
        n, off, src, dst, kind = graphgen.batch(10_000, seed=3)
        lines.append("# g <index> <n> <m> <triangles> <4-truss edges>  (batch of 10,000, seed 3)")
        for i in batch_sample(n):
            og = oracle.OracleGraph.from_edges(src[off[i]:off[i + 1]], dst[off[i]:off[i + 1]],
                                               int(n[i]))
            lines.append(f"g {i} {n[i]} {og.m} {og.count()} {og.ktruss(4)[2]}")
            og.close()
    elif name == "serve_pool":
        pool = graphgen.rmat_pool(64, seed=4)
        lines.append("# g <id> <n> <m> <triangles> <k-truss edges for k = 3 .. 8>  (pool of 64, seed 4)")
        for gid, (s, d, nv) in pool.items():
            og = oracle.OracleGraph.from_edges(s, d, nv)
            sizes = og.truss_levels(8)
            lines.append(f"g {gid} {nv} {og.m} {og.count()} " + " ".join(map(str, sizes)))
            og.close()
            print(lines[-1], f"({time.time() - t0:.1f} s)", flush=True)
    else:
        raise SystemExit(f"unknown set {name}")
    lines.append(f"# oracle wall time {time.time() - t0:.1f} s")
    out = os.path.join(HERE, f"{name}_oracle.txt")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    print(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--truss", action="store_true", help="also the full truss decomposition")
    ap.add_argument("--ks", default="", help="comma-separated k values for single k-truss runs")
    args = ap.parse_args()
    if args.workload in ("batch10k_sample", "serve_pool"):
        many_graphs(args.workload)
        return
    w = graphgen.WORKLOADS[args.workload]
    s, d, n = w.generate()
    lines = [f"# oracle results for workload {w.name}: {w.description}",
             "# written by tests/golden/make_oracle_fixtures.py (oracle only)"]
    out = os.path.join(HERE, f"{w.name}_oracle.txt")
    t0 = time.time()

    def checkpoint():
        with open(out + ".partial", "w") as f:
            f.write("\n".join(lines) + f"\n# partial, {time.time() - t0:.1f} s so far\n")
        print(lines[-1], f"({time.time() - t0:.1f} s)", flush=True)

    g = oracle.OracleGraph.from_edges(s, d, n)
    lines.append(f"n {n}")
    lines.append(f"m_in {len(s)}")
    lines.append(f"m {g.m}")
    lines.append(f"lo_hi_sha256 {sha(g.lo)} {sha(g.hi)}")
    checkpoint()
    T = g.count()
    lines.append(f"triangles {T}")
    checkpoint()
    sup = g.support()
    lines.append(f"support_sha256 {sha(sup)}")
    lines.append(f"support_sum {int(sup.sum(dtype=np.int64))}")
    checkpoint()
    for k in [int(x) for x in args.ks.split(",") if x]:
        mask, _, left = g.ktruss(k)
        lines.append(f"ktruss {k} {left} {sha(mask.astype(np.int32))}")
        checkpoint()
    if args.truss:
        kmax, t = g.truss_decomposition()
        lines.append(f"kmax {kmax}")
        lines.append(f"truss_sha256 {sha(t)}")
        counts = [int((t >= k).sum()) for k in range(2, kmax + 2)]
        lines.append("truss_edges_from_k2 " + " ".join(map(str, counts)))
    lines.append(f"# oracle wall time {time.time() - t0:.1f} s")
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")
    if os.path.exists(out + ".partial"):
        os.remove(out + ".partial")
    print(out)


if __name__ == "__main__":
    main()
