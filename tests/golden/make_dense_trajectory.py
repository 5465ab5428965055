"""Write the FP64 oracle's relative-error trajectory of a dense planted problem.

Runs the oracle (``oracle/method.py``: Alg. 1 with the sketched subproblems of
Section 3.2, one projected-gradient step per half, eq. gradient_descent) for T
outer iterations from the default Philox initial factors and records
||M - U V^T||_F / ||M||_F (Section 5.1) after every iteration.  Only the
oracle and the shared input generator (``synthdata``) are called; nothing
comes from the GPU library.

Default: the dense image-like precision study, planted 65,536 x 16,384
(k = 64, 70 % zeroed factors, |N(0, 0.01^2)| noise, seed 0), Gaussian sketch
d = d' = 2048, alpha = beta = 1, T = 100.  On 8 x86 cores one iteration takes
about half a minute (8.8 TFLOP in FP64), so the run checkpoints (U, V, t and
the errors so far) after every iteration into ``_ckpt/`` beside this file
and resumes from there.

    python tests/golden/make_dense_trajectory.py            # full run
    python tests/golden/make_dense_trajectory.py --m 2048 --n 1024 --k 16 --d 128 --T 5
"""
import argparse
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import method  # noqa: E402
from synthdata import planted_dense  # noqa: E402


def _sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=65536)
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--k", type=int, default=64)
    ap.add_argument("--d", type=int, default=2048)
    ap.add_argument("--T", type=int, default=100)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--zero-frac", type=float, default=0.7)
    ap.add_argument("--noise", type=float, default=0.01)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    m, n, k, d, T, seed = args.m, args.n, args.k, args.d, args.T, args.seed
    name = "dense_%dx%d_k%d_d%d_gaussian_pgd_T%d" % (m, n, k, d, T)
    out = args.out or os.path.join(HERE, name + ".json")
    ckdir = os.path.join(HERE, "_ckpt")
    os.makedirs(ckdir, exist_ok=True)
    ck = os.path.join(ckdir, name + ".npz")

    M32, _, _ = planted_dense(m, n, k, seed, zero_frac=args.zero_frac, noise=args.noise)
    M = M32.astype(np.float64)
    del M32
    MT = np.ascontiguousarray(M.T)
    opt = method.Options(sketch=method.GAUSSIAN, d=d)
    if os.path.exists(ck):
        z = np.load(ck)
        U, V, t0, errs = z["U"], z["V"], int(z["t"]), list(z["errs"])
        secs = list(z["secs"])
    else:
        U0, V0 = method.default_init(seed, m, n, k)
        U, V, t0, errs, secs = U0.astype(np.float64), V0.astype(np.float64), 0, [], []
    for t in range(t0, T):
        a = time.time()
        U, V = method.outer_iteration(M, MT, U, V, seed, t, opt)
        errs.append(method.rel_error(M, U, V))
        secs.append(time.time() - a)
        np.savez(ck + ".tmp.npz", U=U, V=V, t=t + 1, errs=np.array(errs), secs=np.array(secs))
        os.replace(ck + ".tmp.npz", ck)
        print("t=%d err=%.9f %.1fs" % (t, errs[-1], secs[-1]), flush=True)
    rec = {
        "what": "FP64 oracle relative error ||M - U V^T||_F / ||M||_F after each outer iteration "
                "(Alg. 1, sketched subproblems of Section 3.2, one PGD step per half, eq. gradient_descent; "
                "error of Section 5.1)",
        "written_by": "tests/golden/make_dense_trajectory.py (calls oracle/ and synthdata only)",
        "input": {"recipe": "synthdata.planted_dense", "m": m, "n": n, "k": k, "seed": seed,
                  "zero_frac": args.zero_frac, "noise": args.noise},
        "method": {"sketch": "gaussian", "d": d, "d_v": d, "solver": "pgd", "alpha": 1.0, "beta": 1.0,
                   "power_iters": 32, "init": "default Philox streams 2 and 3", "T": T},
        "oracle_sources": {"oracle/method.py": _sha(os.path.join(ROOT, "oracle", "method.py")),
                           "oracle/rng.c": _sha(os.path.join(ROOT, "oracle", "rng.c"))},
        "errors": [float(e) for e in errs],
        "seconds_per_iteration": float(np.median(secs)) if secs else None,
        "host_cores": os.cpu_count(),
    }
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
