"""The oracle built with -fopenmp (the CPU baseline on all host cores: one
parallel loop over each colour step's rows and each SpMV's rows) computes the
same bits as the plain single-threaded build: every row's arithmetic is the
same sequence of operations, only the rows are shared among threads."""
import numpy as np
import pytest

from hpcg_inputs import normal
from oracle import OracleProblem, load_omp


@pytest.fixture(scope="module")
def omp():
    try:
        return load_omp()
    except Exception as e:  # noqa: BLE001 - a compiler without OpenMP
        pytest.skip("no OpenMP in this compiler: %s" % e)


@pytest.mark.parametrize("dims,levels", [((16, 16, 16), 4), ((24, 8, 16), 3)])
def test_openmp_build_gives_the_same_bits(omp, dims, levels):
    n = int(np.prod(dims))
    a = OracleProblem(*dims, levels=levels)
    b = OracleProblem(*dims, levels=levels, lib=omp)
    x = normal(n, 201)
    np.testing.assert_array_equal(a.spmv(x), b.spmv(x))
    np.testing.assert_array_equal(a.rbgs(x, np.zeros(n)), b.rbgs(x, np.zeros(n)))
    np.testing.assert_array_equal(a.mg(x), b.mg(x))
    rhs = a.rhs()
    xa, ha = a.pcg(rhs, max_iters=12, tol=0.0)
    xb, hb = b.pcg(rhs, max_iters=12, tol=0.0)
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ha, hb)
