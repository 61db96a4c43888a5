"""Write the whole-history digests of the full-size single solves.

Each file records what the CPU oracle computes for one workload -- classic
PBiCGStab (Fig. 2) or pipelined p-PBiCGStab (Fig. 4) with Jacobi, x0 = 0,
b = A*1 (the oracle's own SpMV), tol 1e-10 -- so that the GPU test can compare
its whole run bit for bit without spending minutes in the oracle (the method
of Sec. 5.3: every iterate of the reproducible solver against a sequential
reference). Only `oracle/` computes these values; nothing here comes from
the CUDA library.

Recorded per workload: the iteration count, status and the scalars of
rbs_info as binary64 hex; sha256 of the whole history (iters x 12 binary64,
NaN fields canonicalised to 0x7ff8000000000000); tau of every iteration in hex
(to locate a first difference); sha256 of x and x at a few fixed indices.

    python tests/golden/make_c3_digests.py [name ...]

Workloads: poisson256_{classic,pipelined} (Poisson 7-point 256^3) and
convdiff192_{classic,pipelined} (first-order upwind convection-diffusion
192^3, Peclet 10, velocity (1,1,1)).
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

TOL = 1e-10
MAXIT = 20000
QNAN = np.uint64(0x7FF8000000000000)
WORKLOADS = {
    "poisson256_classic": ("poisson3d", (256,), 0),
    "poisson256_pipelined": ("poisson3d", (256,), 1),
    "convdiff192_classic": ("convdiff3d", (192, 10.0), 0),
    "convdiff192_pipelined": ("convdiff3d", (192, 10.0), 1),
}
X_SAMPLES = (0, 1, 4097, 65537, 1000003, 4000037)


def canonical_bits(a) -> np.ndarray:
    """binary64 bits with every NaN replaced by the quiet NaN 0x7ff8000000000000."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    bits = a.view(np.uint64).copy()
    bits[np.isnan(a)] = QNAN
    return bits


def history_sha(hist) -> str:
    return hashlib.sha256(canonical_bits(hist).tobytes()).hexdigest()


def x_sha(x) -> str:
    return hashlib.sha256(np.ascontiguousarray(x, dtype=np.float64).tobytes()).hexdigest()


def hx(v: float) -> str:
    return f"{int(canonical_bits(np.array([v]))[0]):016x}"


def path(name: str) -> str:
    return os.path.join(HERE, f"c3_{name}.txt")


def write(name: str) -> None:
    import oracle
    from paper_2302_04180_gb300 import gen
    oracle.build()
    fn, args, variant = WORKLOADS[name]
    A = getattr(gen, fn)(*args)
    b = oracle.spmv(A, np.ones(A.n))
    t = time.time()
    o = oracle.solve(A, b, tol=TOL, maxit=MAXIT, variant=variant)
    dt = time.time() - t
    tau_col = 7 if variant == 0 else 8
    lines = [
        f"# {name}: oracle {'classic PBiCGStab (Fig. 2)' if variant == 0 else 'pipelined p-PBiCGStab (Fig. 4)'},",
        f"# {fn}{args}, n = {A.n}, nnz = {A.nnz}, Jacobi, x0 = 0, b = A*1, tol = {TOL:g}",
        "# written by tests/golden/make_c3_digests.py from oracle/ only "
        f"({dt:.0f} s); compared bit for bit by tests/test_gpu_full_history.py",
        f"iters {o['iters']}",
        f"status {o['status']}",
        f"converged {o['converged']}",
    ]
    for k in ("tau0", "tau_final", "rho0", "tau_max", "alpha0", "mu0"):
        lines.append(f"{k} {hx(o[k])}")
    lines.append(f"history_sha256 {history_sha(o['hist'])}")
    lines.append(f"x_sha256 {x_sha(o['x'])}")
    for i in X_SAMPLES:
        if i < A.n:
            lines.append(f"x {i} {hx(o['x'][i])}")
    for j in range(o["iters"]):
        lines.append(f"tau {j} {hx(o['hist'][j, tau_col])}")
    with open(path(name), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"{name}: {o['iters']} iterations, {dt:.0f} s", flush=True)


def read(name: str) -> dict:
    d = {"x": {}, "tau": {}}
    for line in open(path(name)):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] in ("x", "tau"):
            d[f[0]][int(f[1])] = f[2]
        else:
            d[f[0]] = f[1]
    return d


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(WORKLOADS):
        write(nm)
