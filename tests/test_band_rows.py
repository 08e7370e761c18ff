"""Host logic of the factorisation launches: the rows and columns a partial-Cholesky launch
visits (interior band, interface-row profile, identity block; BandRows in csrc/common.cuh) must
include every row whose L entries in the launch's K range are not structurally zero.  Checked
against the nonzero pattern of L computed by a dense FP64 Cholesky of random matrices with that
structure (structural zeros of L are exact zeros in floating point), through a host-only build
of the same header."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from conftest import ROOT

CSRC = os.path.join(ROOT, "paper_2101_02959_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("band") / "band_rows")
    src = os.path.join(ROOT, "tests", "native", "band_rows_harness.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-gencode", "arch=compute_103a,code=sm_103a", src,
                        "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _query(exe, m, e, band, id0, q, queries):
    lines = [f"{m} {e} {band} {id0} {len(q)}", " ".join(str(int(x)) for x in q), str(len(queries))]
    lines += [f"{a} {b}" for a, b in queries]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    out = []
    for ln in r.stdout.strip().splitlines():
        v = [int(x) for x in ln.split()]
        out.append((v[0], v[2:2 + v[1]]))
    return out


def _structure(rng, e, band, n_iface, identity):
    """Random SPD interior block with half-bandwidth `band`, interface rows coupled from a
    non-decreasing first column on, and (identity=True) an identity block below them.
    Returns the matrix rows below e, the L pattern over columns [0, e) and the profile."""
    A = np.zeros((e, e))
    for i in range(e):
        for k in range(max(0, i - band), i):
            if rng.random() < 0.4:
                A[i, k] = A[k, i] = rng.standard_normal()
    A += np.eye(e) * (np.abs(A).sum(1).max() + 1.0)
    first = np.sort(rng.integers(0, e + 5, n_iface))
    G = np.zeros((n_iface, e))
    for g in range(n_iface):
        f = int(first[g])
        if f < e:
            cols = np.unique(np.concatenate([[f], rng.integers(f, min(e, f + 2 * band + 3), 4)]))
            G[g, cols] = rng.standard_normal(len(cols))
    below = [G] + ([np.eye(e)] if identity else [])
    B = np.vstack(below)
    L11 = np.linalg.cholesky(A)
    L21 = np.linalg.solve(L11, B.T).T
    L = np.vstack([L11, L21])
    q = np.minimum(first, e).astype(int)
    for g in range(n_iface - 2, -1, -1):
        q[g] = min(q[g], q[g + 1])
    return L != 0.0, q


@pytest.mark.parametrize("e,band,n_iface,identity,profile", [
    (300, 25, 120, False, True), (300, 25, 120, False, False), (200, 1 << 30, 60, True, False),
    (260, 40, 0, True, False), (129, 7, 33, False, True)])
def test_launch_rows_cover_every_nonzero_row(harness, e, band, n_iface, identity, profile):
    rng = np.random.default_rng(e + n_iface)
    nz, q = _structure(rng, e, min(band, e), n_iface, identity)
    m = nz.shape[0]
    id0 = e + n_iface if identity else 1 << 30
    queries = []
    for ke in sorted(set([1, 5, 64, 128, 129, 200, e - 1, e]) & set(range(1, e + 1))):
        for row0 in sorted(set([ke, min(e, ke + 3), e])):
            queries.append((row0, ke))
    got = _query(harness, m, e, band, id0, q if profile else [], queries)
    for (row0, ke), (lim, rows) in zip(queries, got):
        rows = np.array(rows, int)
        assert len(set(rows.tolist())) == len(rows) and (rows >= row0).all() and (rows < m).all()
        need = [r for r in range(row0, m) if nz[r, :ke].any()]
        assert set(need) <= set(rows.tolist()), (row0, ke)
        # columns of a trailing update: every interior column whose L row reaches below ke
        need_c = [c for c in range(ke, e) if nz[c, :ke].any()]
        assert all(c < lim for c in need_c), (ke, lim)
        if band < e and not profile:  # the band is used: interior rows past ke + band are left out
            assert all(r >= e or r < ke + band for r in rows)
    if profile:
        # the final update of later rows g.. starts at ifirst[g] rounded down to 4 columns
        for g in range(0, n_iface, 7):
            assert not nz[e + g:e + n_iface, :q[g] & ~3].any()


def test_dense_descriptor_visits_every_row(harness):
    got = _query(harness, 50, 30, 1 << 30, 1 << 30, [], [(10, 10), (30, 30)])
    assert got[0] == (30, list(range(10, 50)))
    assert got[1] == (30, list(range(30, 50)))
