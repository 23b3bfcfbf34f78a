#!/usr/bin/env python3
"""Write the exact kNN graph of the 70000 x 784 MNIST-shaped workload.

The graph (k = 5, Section 4.2: the k nearest points q != p by Euclidean
distance, ascending by (distance, index)) is computed by the FP64 oracle
alone -- nothing from the CUDA path -- and stored with the SHA-256 of the
float32 input it was computed on, so a test can check that it regenerated
the same points.  The squared distances are not stored: the oracle
recomputes them for the stored pairs (``oracle.pair_d2``).

  python tests/golden/make_mnist_like_knn.py     # about 15 min on 8 cores
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1810_13044_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "mnist_like_70000x784_k5_knn.npz")
K = 5


def main():
    X, _ = inputs.mnist_like()
    sha = hashlib.sha256(np.ascontiguousarray(X).tobytes()).hexdigest()
    t0 = time.perf_counter()
    idx, _ = oracle.knn(X, K)
    secs = time.perf_counter() - t0
    np.savez_compressed(OUT, idx=idx.astype(np.int32), x_sha256=np.array(sha), k=np.array(K))
    print(f"wrote {OUT}: {idx.shape}, {secs:.0f} s on {oracle.threads()} threads, X sha256 {sha}")


if __name__ == "__main__":
    main()
