"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/hpcg_oracle.c (a dropped
term, a wrong sign, index or loop order), compiles it on the CPU, and checks
that at least one pin (closed forms, dense textbook routines, dense solves)
fails for the mutant while every pin holds for the real oracle.
"""
import os
import tempfile

import numpy as np
import pytest

from oracle import OracleProblem
from oracle.oracle import compile_source, load_library, source_path
from tests import dense_ref as D


def _close(a, b, tol):
    return np.all(np.isfinite(a)) and np.abs(a - b).max() <= tol * max(np.abs(b).max(), 1e-300)


def _pins(lib):
    """Every pin as (name, bool); exceptions count as a failed pin."""
    out = []

    def pin(name, fn):
        try:
            out.append((name, bool(fn())))
        except Exception:  # a mutant may crash a pin (e.g. a non-SPD matrix)
            out.append((name, False))

    rng = np.random.default_rng(0)

    def operator():
        kappa = np.linspace(0.0, 1.0, 60)
        p = OracleProblem(3, 4, 5, levels=1, kappa=kappa, lib=lib)
        return np.array_equal(p.csr().toarray(), D.kron_operator(3, 4, 5, kappa=kappa)) and \
            p.nnz() == (3 * 3 - 2) * (3 * 4 - 2) * (3 * 5 - 2)

    def colouring():
        p = OracleProblem(4, 4, 4, levels=1, lib=lib)
        A = p.csr().tocoo()
        off = A.row != A.col
        col = p.colors()
        return np.all(col[A.row[off]] != col[A.col[off]]) and np.array_equal(col, D.parity_colors(4, 4, 4))

    def forward_sweep():
        p = OracleProblem(4, 4, 4, levels=1, symmetric=False, lib=lib)
        A = p.csr().toarray()
        r, z0 = rng.standard_normal(64), rng.standard_normal(64)
        return _close(p.rbgs(r, z0), D.gs_forward_sorted(A, D.parity_colors(4, 4, 4), r, z0), 1e-12)

    def symmetric_sweep():
        p = OracleProblem(3, 5, 7, levels=1, lib=lib)
        A = p.csr().toarray()
        cols = D.parity_colors(3, 5, 7)
        r, z0 = rng.standard_normal(105), rng.standard_normal(105)
        ref = D.gs_backward_sorted(A, cols, r, D.gs_forward_sorted(A, cols, r, z0))
        return _close(p.rbgs(r, z0), ref, 1e-12)

    def colour_step_residual():
        p = OracleProblem(4, 4, 4, levels=1, lib=lib)
        A = p.csr().toarray()
        r, z = rng.standard_normal(64), rng.standard_normal(64)
        cols = D.parity_colors(4, 4, 4)
        zn = p.rbgs_color_step(3, r, z)
        res = r - A @ zn
        return np.abs(res[cols == 3]).max() < 1e-12 * 30 and np.array_equal(zn[cols != 3], z[cols != 3])

    def transfers():
        p = OracleProblem(8, 8, 8, levels=3, lib=lib)
        ok = True
        for l in range(2):
            f2c = p.f2c(l)
            nxf, nyf, _ = p.dims(l)
            nxc, nyc, _ = p.dims(l + 1)
            c = np.arange(len(f2c))
            ok &= np.array_equal(f2c % nxf, 2 * (c % nxc)) and np.array_equal((f2c // nxf) % nyf, 2 * ((c // nxc) % nyc))
            R = D.injection_matrix(p.n(l), f2c)
            v, zc, z = rng.standard_normal(p.n(l)), rng.standard_normal(p.n(l + 1)), rng.standard_normal(p.n(l))
            ok &= np.array_equal(p.restrict(v, l), R @ v) and _close(p.prolong_add(zc, z, l), z + R.T @ zc, 0)
        return ok

    def vcycle():
        ok = True
        for kappa in (None, np.random.default_rng(3).uniform(0, 1, 512)):
            p = OracleProblem(8, 8, 8, levels=3, kappa=kappa, lib=lib)
            As = [p.csr(l).toarray() for l in range(3)]
            Rs = [D.injection_matrix(p.n(l), p.f2c(l)) for l in range(2)]
            cols = [D.parity_colors(*p.dims(l)) for l in range(3)]
            # the dense reference uses the generator's own coarse operators: also
            # check them against the closed form (regenerated stencil, injected kappa)
            kap_c = None if kappa is None else kappa[p.f2c(0)]
            ok &= np.array_equal(As[1], D.kron_operator(4, 4, 4, kappa=kap_c))
            r = rng.standard_normal(512)
            ok &= _close(p.mg(r), D.dense_vcycle(As, cols, Rs, r), 1e-11)
        return ok

    def coarse_inputs():
        # forward-only sweep: the restricted residual is then not rounding noise
        p = OracleProblem(8, 8, 8, levels=3, symmetric=False, lib=lib)
        As = [p.csr(l).toarray() for l in range(3)]
        cols = [D.parity_colors(*p.dims(l)) for l in range(3)]
        Rs = [D.injection_matrix(p.n(l), p.f2c(l)) for l in range(2)]
        p.mg(rng.standard_normal(512))
        r = rng.standard_normal(512)
        p.mg(r)
        ok = True
        for l in (1, 2):
            z = D.gs_forward_sorted(As[l - 1], cols[l - 1], r, np.zeros(p.n(l - 1)))
            rc = Rs[l - 1] @ (r - As[l - 1] @ z)
            rc_o, zc_o = p.coarse_state(l)
            zc = D.dense_vcycle(As[l:], cols[l:], Rs[l:], rc, symmetric=False)
            ok &= _close(rc_o, rc, 1e-12) and _close(zc_o, zc, 1e-12)
            r = rc
        return ok

    def krylov():
        p = OracleProblem(4, 4, 4, levels=2, lib=lib)
        A = D.kron_operator(4, 4, 4)
        n = 64
        M = np.zeros((n, n))
        for j in range(n):
            e = np.zeros(n)
            e[j] = 1.0
            M[:, j] = p.mg(e)
        M = 0.5 * (M + M.T)
        b = rng.standard_normal(n)
        xs = np.linalg.solve(A, b)
        ok = True
        for k in (1, 2, 3):
            xk, _ = p.pcg(b, max_iters=k, tol=0.0)
            V = [M @ b]
            with np.errstate(all="ignore"):  # mutants may overflow here
                for _ in range(k - 1):
                    V.append(M @ (A @ V[-1]))
            Q, _ = np.linalg.qr(np.array(V).T)
            xm = Q @ np.linalg.solve(Q.T @ A @ Q, Q.T @ b)
            e = xk - xm
            ok &= np.sqrt(e @ A @ e) <= 1e-9 * np.sqrt(xs @ A @ xs)
        return ok

    def history_and_stop():
        # hist[k-1] is the true relative residual of the k-th iterate, and the
        # solve stops at the first k where it reaches the tolerance
        p = OracleProblem(4, 6, 8, levels=2, lib=lib)
        A = D.kron_operator(4, 6, 8)
        b = rng.standard_normal(p.n())
        _, hist = p.pcg(b, max_iters=40, tol=1e-6)
        ok = 0 < len(hist) < 40 and hist[-1] <= 1e-6 and np.all(hist[:-1] > 1e-6)
        for k in range(1, len(hist) + 1):
            xk, _ = p.pcg(b, max_iters=k, tol=0.0)
            ok &= abs(np.linalg.norm(b - A @ xk) / np.linalg.norm(b) - hist[k - 1]) <= 1e-12
        return ok

    def direct_solve():
        p = OracleProblem(4, 6, 8, levels=2, lib=lib)
        A = D.kron_operator(4, 6, 8)
        b = rng.standard_normal(p.n())
        x, _ = p.pcg(b, max_iters=100, tol=1e-14)
        xo, _ = p.pcg(A @ np.ones(p.n()), max_iters=100, tol=1e-14)
        return _close(x, np.linalg.solve(A, b), 1e-11) and np.abs(xo - 1).max() < 1e-11

    for name, fn in [("operator", operator), ("colouring", colouring), ("forward_sweep", forward_sweep),
                     ("symmetric_sweep", symmetric_sweep), ("colour_step", colour_step_residual),
                     ("transfers", transfers), ("vcycle", vcycle), ("coarse_inputs", coarse_inputs), ("krylov", krylov), ("history_and_stop", history_and_stop),
                     ("direct_solve", direct_solve)]:
        pin(name, fn)
    return out


# one plausible mistake per case: (name, text in the oracle, replacement)
MUTANTS = [
    ("off-diagonal sign", "vals[cnt] = -1.0;", "vals[cnt] = 1.0;"),
    ("diagonal value", "vals[cnt] = 26.0 + (kappa ? kappa[i] : 0.0);", "vals[cnt] = 27.0 + (kappa ? kappa[i] : 0.0);"),
    ("kappa sign", "vals[cnt] = 26.0 + (kappa ? kappa[i] : 0.0);", "vals[cnt] = 26.0 - (kappa ? kappa[i] : 0.0);"),
    ("dropped +x neighbour", "for (int dx = -1; dx <= 1; ++dx) {\n        int xx", "for (int dx = -1; dx <= 0; ++dx) {\n        int xx"),
    ("greedy looks ahead", "if (j != i && L->color[j] >= 0", "if (j > i && L->color[j] >= 0"),
    ("update sign", "double v = r[i] - tmp[i] + z[i] * d;", "double v = r[i] + tmp[i] + z[i] * d;"),
    ("update drops diagonal", "double v = r[i] - tmp[i] + z[i] * d;", "double v = r[i] - tmp[i];"),
    ("colour step updates every row", "  for (long i = 0; i < L->n; ++i) {\n    if (L->color[i] != k) continue;\n    double d",
     "  for (long i = 0; i < L->n; ++i) {\n    double d"),
    ("backward sweep in forward order", "for (int k = L->ncolors - 1; k >= 0; --k) orc_rbgs_color_step",
     "for (int k = 0; k < L->ncolors; ++k) orc_rbgs_color_step"),
    ("injection from odd corner", "long f = 2L * xc + (long)nfx", "long f = 2L * xc + 1 + (long)nfx"),
    ("refinement overwrites", "z[F->f2c[c]] = z[F->f2c[c]] + zc[c];", "z[F->f2c[c]] = zc[c];"),
    ("restriction of r, not r - Az", "L->tmp[i] = r[i] - L->f[i];", "L->tmp[i] = r[i];"),
    ("coarse kappa not injected", "kc[c] = kap[F->f2c[c]];", "kc[c] = kap[c];"),
    ("no post-smoothing", "orc_rbgs(p, l, r, z);                       /* post-smoothing */", "/* none */"),
    ("coarse z not reset", "for (long c = 0; c < C->n; ++c) C->z[c] = 0.0; /* z_c <- 0 */", "/* none */"),
    ("beta sign", "pp[i] = z[i] + beta * pp[i];", "pp[i] = z[i] - beta * pp[i];"),
    ("alpha from p.p", "double alpha = rtz / dot(n, pp, Ap);", "double alpha = rtz / dot(n, pp, pp);"),
    ("dot drops last term", "for (long i = 0; i < n; ++i) s += a[i] * b[i];", "for (long i = 0; i + 1 < n; ++i) s += a[i] * b[i];"),
    ("beta from the updated r.z", "double beta = rtz_new / rtz;\n      rtz = rtz_new;", "rtz = rtz_new;\n      double beta = rtz_new / rtz;"),
    ("x update sign", "x[i] = x[i] + alpha * pp[i];", "x[i] = x[i] - alpha * pp[i];"),
    ("r updated with p, not Ap", "r[i] = r[i] - alpha * Ap[i];", "r[i] = r[i] - alpha * pp[i];"),
    ("history not relative", "double rel = sqrt(dot(n, r, r)) / normr0;", "double rel = sqrt(dot(n, r, r));"),
    ("never stops on tolerance", "if (rel <= tol) break;", "if (rel < 0.0) break;"),
    ("residual sign", "for (long i = 0; i < n; ++i) r[i] = b[i] - Ap[i];", "for (long i = 0; i < n; ++i) r[i] = Ap[i] - b[i];"),
]


@pytest.fixture(scope="module")
def workdir():
    with tempfile.TemporaryDirectory() as d:
        yield d


def test_all_pins_hold_for_the_oracle():
    from oracle.oracle import _load
    failed = [name for name, ok in _pins(_load()) if not ok]
    assert not failed, failed


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(name, old, new, workdir):
    src = open(source_path()).read()
    assert src.count(old) >= 1, "mutation anchor missing: %s" % name
    mutated = src.replace(old, new, 1)
    path = os.path.join(workdir, "m_%d.c" % abs(hash(name)))
    with open(path, "w") as f:
        f.write(mutated)
    lib = load_library(compile_source(path, path[:-2] + ".so"))
    results = _pins(lib)
    assert not all(ok for _, ok in results), "no pin caught: %s" % name
