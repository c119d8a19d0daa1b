"""Dense numpy helpers for the tests (independent of the oracle and the library)."""
import numpy as np

import graphgen as gg


def dense_laplacian(g: gg.Graph) -> np.ndarray:
    """A = L_w + diag(d) straight from Eq. (1): A_ii = sum_j w_ij + d_i, A_ij = -w_ij."""
    n = g.n
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(g.rowptr))
    A[rows, g.col] = -g.w
    A[np.arange(n), np.arange(n)] = -A.sum(axis=1)
    if g.d is not None:
        A[np.arange(n), np.arange(n)] += g.d
    return A


def prolongation(agg: np.ndarray, nH: int) -> np.ndarray:
    """Piecewise-constant P: column l is the indicator of aggregate l."""
    P = np.zeros((agg.size, nH))
    P[np.arange(agg.size), agg] = 1.0
    return P


def random_graph(n: int, p: float, seed: int, wmax: int = 1, d_frac: float = 0.0, connected=True) -> gg.Graph:
    """Erdos-Renyi-like graph with integer weights in [1, wmax]; a spanning path keeps it connected."""
    rng = np.random.default_rng(seed)
    edges = set()
    if connected:
        perm = rng.permutation(n)
        for a, b in zip(perm[:-1], perm[1:]):
            edges.add((min(a, b), max(a, b)))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < p:
                edges.add((i, j))
    e = np.array(sorted(edges), dtype=np.int64).reshape(-1, 2)
    w = rng.integers(1, wmax + 1, size=len(e)).astype(np.float64)
    d = None
    if d_frac > 0:
        d = np.where(rng.random(n) < d_frac, rng.integers(1, 4, size=n).astype(np.float64), 0.0)
        if not d.any():
            d[0] = 1.0
    return gg.csr_from_edges(n, e[:, 0], e[:, 1], w, d, name=f"rand{n}_{seed}")


def path_graph(n: int) -> gg.Graph:
    i = np.arange(n - 1)
    return gg.csr_from_edges(n, i, i + 1, name=f"path{n}")


def complete_graph(n: int) -> gg.Graph:
    i, j = np.triu_indices(n, 1)
    return gg.csr_from_edges(n, i, j, name=f"K{n}")


def star_graph(n: int) -> gg.Graph:
    return gg.csr_from_edges(n, np.zeros(n - 1, np.int64), np.arange(1, n), name=f"star{n}")


def cheb_q(coef: np.ndarray, l0: float, l1: float, x: np.ndarray) -> np.ndarray:
    """Evaluate sum_j c_j T_j(t(x)), t = (2x - l1 - l0)/(l1 - l0), with numpy's chebval."""
    t = (2.0 * np.asarray(x) - l1 - l0) / (l1 - l0)
    return np.polynomial.chebyshev.chebval(t, coef)


def matrix_function(A: np.ndarray, f) -> np.ndarray:
    lam, V = np.linalg.eigh(A)
    return (V * f(lam)) @ V.T


def sparse_laplacian(g: gg.Graph):
    """A = L_w + diag(d) of Eq. (1) as a scipy CSR matrix."""
    import scipy.sparse as sp

    n = g.n
    W = sp.csr_matrix((g.w, g.col, g.rowptr), shape=(n, n))
    deg = np.asarray(W.sum(axis=1)).ravel()
    if g.d is not None:
        deg = deg + g.d
    return (sp.diags(deg) - W).tocsr()


def c_struct_layouts(include_dir: str, header: str, structs, workdir) -> dict:
    """{(struct, field): offset, (struct, 'sizeof'): size} as a C compiler lays
    out `structs` (pairs of C name and ctypes class, whose field names are the
    C member names) from `header`; None if no C compiler is available."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        return None
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{header}"', "int main(void) {"]
    for name, cls in structs:
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    src = workdir / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = workdir / "layout"
    subprocess.run([cc, "-std=c99", "-I", include_dir, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return {(a, b): int(c) for a, b, c in (ln.split() for ln in out.splitlines())}


def assert_layouts_match(layout: dict, structs):
    import ctypes as C

    for name, cls in structs:
        assert layout[(name, "sizeof")] == C.sizeof(cls), name
        for f, _ in cls._fields_:
            assert layout[(name, f)] == getattr(cls, f).offset, (name, f)


def restarted_pcg(A, B, b, R, iters):
    """Textbook preconditioned CG (z = B r, beta = r'z / r_old'z_old), the
    search direction reset to z at every multiple of R iterations."""
    x = np.zeros_like(b); r = b.copy(); hist = [1.0]
    p = rz_old = None
    for it in range(iters):
        z = B @ r
        rz = r @ z
        p = z.copy() if it % R == 0 else z + rz / rz_old * p
        Ap = A @ p
        a = rz / (p @ Ap)
        x += a * p
        r -= a * Ap
        rz_old = rz
        hist.append(np.linalg.norm(r) / np.linalg.norm(b))
    return np.array(hist)
