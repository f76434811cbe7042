"""The lambda path's subsample bookkeeping (csrc/subsamples.h), compiled on
the host with g++: each bootstrap sample becomes its distinct rows, ascending,
row j scaled by sqrt(K c_j / n_s), so that the scaled rows give the same
S = X^T X / n as the sample (Eq. 3.2 sees the data only through S)."""
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include <vector>
#include "subsamples.h"
int main() {
  long long n, ns;
  if (std::scanf("%lld %lld", &n, &ns) != 2) return 2;
  std::vector<int64_t> off(ns + 1);
  for (auto& o : off) {
    long long v;
    if (std::scanf("%lld", &v) != 1) return 2;
    o = v;
  }
  std::vector<int32_t> rows(off[ns] > 0 ? off[ns] : 0);
  for (auto& r : rows) {
    long long v;
    if (std::scanf("%lld", &v) != 1) return 2;
    r = (int32_t)v;
  }
  accord::Subsamples S;
  const int st = accord::compress_subsamples(rows.data(), off.data(), ns, n, S);
  std::printf("%d %lld\n", st, (long long)S.kmax);
  if (st != ACCORD_OK) return 0;
  for (size_t i = 0; i < S.off.size(); ++i) std::printf("%lld ", (long long)S.off[i]);
  std::printf("\n");
  for (size_t i = 0; i < S.rows.size(); ++i) std::printf("%d %.17g\n", S.rows[i], S.scale[i]);
  for (double v : S.n_obs) std::printf("%.17g ", v);
  std::printf("\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness():
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "h.cpp"), os.path.join(d, "h")
    open(src, "w").write(HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O2", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_2412_11554_gb300", "csrc"),
                    "-o", exe, src], check=True)
    return exe


def run(exe, n, subs):
    offs = np.concatenate([[0], np.cumsum([len(s) for s in subs])]).astype(np.int64)
    rows = np.concatenate(subs).astype(np.int64) if subs else np.zeros(0, np.int64)
    inp = f"{n} {len(subs)}\n" + " ".join(map(str, offs)) + "\n" + " ".join(map(str, rows)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    st, kmax = map(int, out[0].split())
    if st != 0:
        return st, None
    off = np.array(out[1].split(), dtype=np.int64)
    body = [ln.split() for ln in out[2:2 + off[-1]]]
    r = np.array([int(b[0]) for b in body], dtype=np.int64)
    sc = np.array([float(b[1]) for b in body])
    n_obs = np.array(out[2 + off[-1]].split(), dtype=float)
    return st, dict(kmax=kmax, off=off, rows=r, scale=sc, n_obs=n_obs)


def test_bootstrap_samples_match_unique_counts(harness):
    rng = np.random.Generator(np.random.PCG64(31))
    n = 57
    subs = [rng.integers(0, n, size=m) for m in (1, 5, 57, 200)] + [np.arange(n)]
    st, got = run(harness, n, subs)
    assert st == 0
    assert got["kmax"] == max(len(np.unique(s)) for s in subs)
    X = rng.standard_normal((n, 6))
    for s, sub in enumerate(subs):
        lo, hi = got["off"][s], got["off"][s + 1]
        u, c = np.unique(sub, return_counts=True)
        assert np.array_equal(got["rows"][lo:hi], u)
        assert np.array_equal(got["scale"][lo:hi], np.sqrt(len(u) * c.astype(float) / len(sub)))
        assert got["n_obs"][s] == len(sub)
        # the scaled distinct rows give the sample's S
        Z = got["scale"][lo:hi, None] * X[u]
        np.testing.assert_allclose(Z.T @ Z / len(u), X[sub].T @ X[sub] / len(sub), rtol=1e-13, atol=1e-14)


def test_rejects_empty_subsamples_and_bad_indices(harness):
    assert run(harness, 10, [np.array([1, 2]), np.zeros(0, dtype=np.int64)])[0] == -1
    assert run(harness, 10, [np.array([1, 10])])[0] == -1
    assert run(harness, 10, [np.array([-1, 3])])[0] == -1
    # the data set's size costs nothing: an index near 2^31 with n = 2^40
    st, got = run(harness, 1 << 40, [np.array([2 ** 31 - 1, 0, 2 ** 31 - 1])])
    assert st == 0 and list(got["rows"]) == [0, 2 ** 31 - 1] and got["kmax"] == 2
