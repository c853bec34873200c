"""The plan of the tiled triangular solves (tile_plan.h), replayed on the host: the tile lists
and the marks of rows other tiles depend on are exact, the walk (teams taking each tile's rows
round robin, a row waiting only for its own dependencies) never stalls whatever the
interleaving, and it reproduces the sequential substitution exactly. The
neighbour sets are the m nearest previous points of a random ordering (Section 2.1), stored in
Morton order as the library stores them. No GPU."""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2310_12000_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("tile") / "tile_plan_host"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "tile_plan_host.cpp"),
                        "-o", str(out)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)
    return out


def _morton_key(locs, bits=16):
    q = np.minimum((locs * (1 << bits)).astype(np.int64), (1 << bits) - 1)
    key = np.zeros(len(locs), np.int64)
    for b in range(bits):
        key |= ((q[:, 0] >> b) & 1) << (2 * b)
        key |= ((q[:, 1] >> b) & 1) << (2 * b + 1)
    return key


def _neighbours(n, m, seed):
    """ELL of B in Morton storage order: row s lists the storage rows of the m nearest
    previous points (Vecchia order = a random permutation) of its point."""
    rng = np.random.default_rng(seed)
    locs = rng.random((n, 2))
    order = rng.permutation(n)                 # Vecchia position -> point
    storage = np.argsort(_morton_key(locs), kind="stable")
    s_of_point = np.empty(n, np.int64)
    s_of_point[storage] = np.arange(n)
    nbr = -np.ones((n, m), np.int64)
    for i in range(1, n):
        prev = order[:i]
        d2 = np.sum((locs[prev] - locs[order[i]]) ** 2, axis=1)
        k = min(i, m)
        pick = prev[np.lexsort((np.arange(i), d2))[:k]]
        nbr[s_of_point[order[i]], :k] = s_of_point[pick]
    return nbr


@pytest.mark.parametrize("n,m,G", [(1500, 10, 1), (1500, 10, 7), (1500, 10, 152), (1500, 20, 304),
                                   (300, 5, 1000), (40, 0, 8), (2500, 30, 64)])
def test_tile_walk_covers_every_dependency_and_never_stalls(exe, n, m, G):
    nbr = _neighbours(n, m, seed=n + m + G)
    for seed in (1, 2):
        inp = f"{n} {m} {G} {seed}\n" + " ".join(map(str, nbr.ravel())) + "\n"
        r = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, timeout=120)
        assert r.returncode == 0 and r.stdout.split() == ["fwd", "ok", "bwd", "ok"] * 3, r.stdout + r.stderr


@pytest.fixture(scope="module")
def halo_exe(tmp_path_factory):
    out = tmp_path_factory.mktemp("halo") / "halo_plan_host"
    r = subprocess.run(["g++", "-O2", "-std=c++17", "-I", CSRC, os.path.join(HERE, "native", "halo_plan_host.cpp"),
                        "-o", str(out)], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail(r.stdout + r.stderr)
    return out


@pytest.mark.parametrize("n,m,ucap,rmax", [(1500, 10, 438, 512), (2500, 20, 219, 512), (3000, 30, 100, 64),
                                           (500, 5, 8, 3), (40, 0, 4, 512)])
def test_staged_product_plan_places_every_row(halo_exe, n, m, ucap, rmax):
    """The staged products' plan (build_halo_plan): blocks cover the rows in order within the row
    and shared-memory limits, and every own row and dependency entry finds its row in the block's
    list. A limit too small for a row's dependencies is refused (the products then stay unstaged)."""
    nbr = _neighbours(n, m, seed=n + m)
    inp = f"{n} {m} {ucap} {rmax}\n" + " ".join(map(str, nbr.ravel())) + "\n"
    r = subprocess.run([str(halo_exe)], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    out = r.stdout.split("\n")
    assert out[0] == "fwd ok" or (out[0] == "fwd refused" and m + 1 > ucap), r.stdout
    assert out[1] == "bwd ok" or out[1] == "bwd refused", r.stdout
    if ucap >= 200:
        assert out[:2] == ["fwd ok", "bwd ok"], r.stdout
