"""Host-side Rayleigh-Ritz solver of the Lanczos driver (compiled with g++), vs scipy."""
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.linalg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2603_03933_gb300", "csrc", "dense_eig.cuh")

DRIVER = r'''
#include <cstdio>
#include <vector>
#include "dense_eig.cuh"
int main() {
    int k; if (scanf("%d", &k) != 1) return 1;
    std::vector<double> T(k * k), G(k * k);
    for (auto& x : T) if (scanf("%lf", &x) != 1) return 1;
    for (auto& x : G) if (scanf("%lf", &x) != 1) return 1;
    double th; std::vector<double> y;
    if (!lbtr::dense::smallest_generalized(k, T, G, th, y)) { printf("fail\n"); return 0; }
    printf("%.17g\n", th);
    for (double v : y) printf("%.17g\n", v);
    return 0;
}
'''


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("deig")
    src = d / "drv.cpp"
    src.write_text(DRIVER)
    out = d / "drv"
    subprocess.run(["g++", "-O2", "-std=c++17", "-x", "c++", "-I", os.path.dirname(HDR), str(src), "-o", str(out)],
                   check=True)
    return str(out)


def _run(exe, t, g):
    k = t.shape[0]
    inp = f"{k}\n" + " ".join(f"{x:.17g}" for x in t.ravel()) + "\n" + " ".join(f"{x:.17g}" for x in g.ravel())
    res = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split()
    return float(res[0]), np.array([float(v) for v in res[1:]])


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (5, 2), (40, 3), (150, 4)])
def test_smallest_generalized_matches_scipy(exe, k, seed):
    rng = np.random.default_rng(seed)
    # tridiagonal T (as Lanczos produces) and an SPD Gram matrix G
    t = np.diag(rng.standard_normal(k)) + np.diag(rng.uniform(0.1, 1, k - 1), 1) + np.diag(rng.uniform(0.1, 1, k - 1), -1) if k > 1 else np.array([[rng.standard_normal()]])
    t = 0.5 * (t + t.T)
    b = rng.standard_normal((k, k))
    g = b @ b.T / k + np.eye(k)
    th, y = _run(exe, t, g)
    ref = scipy.linalg.eigh(t, g, eigvals_only=True)[0]
    assert abs(th - ref) <= 1e-12 * max(1.0, abs(ref))
    # y is an eigenvector of the pencil
    r = t @ y - th * g @ y
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(t) * np.linalg.norm(y)
