"""Parity at the full size of the benchmark's workloads: the 10,000,000-vertex
random game (out-degree U[2,5], owners p = 0.5, permuted priorities, seed 0),
the 10,000,000-vertex ladder game and the random game with priorities uniform
over 0..3 (count-vector mode), loaded from device arrays and solved to device
arrays through the C ABI, as the benchmark does (the loop as one CUDA graph).

* The final results, element for element: every output array of the full
  solve (winners, both strategies, the dummies' choices, class, depth and
  rank of every valuation) and the iteration counts against the oracle's full
  solve of the same game, stored as SHA-256 digests and sampled values in
  tests/golden/full_size_digests.json by tests/golden/make_full_size_digests.py
  (which calls only the oracle; its solves take minutes on one core, longer
  than a GPU test run may).

* The start of the trajectory, element by element: the profile after the
  first three valuations (the iteration cap) and its valuation, against the
  oracle's after the same three.
* The end, on every vertex: the oracle values the GPU's final profile; that
  valuation equals the GPU's reported one and leaves neither player a
  strictly better edge, which is where Algorithm 1 stops and makes the
  profile optimal (Theorem 1), so the winning regions are certified.

The oracles take about half a minute per game (preprocessing, four
valuations). 20M-vertex games with 3 and 4 priorities (more than 2^24 ids
with the dummies' level) check the count-vector digits sized by level.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import o2, o3
from paper_1705_02313_gb300 import gen

import certificate as cert
from test_gpu_parity import profile_to_original

pytestmark = pytest.mark.gpu

N, DMIN, DMAX, SEED = 10_000_000, 2, 5, 0


@pytest.fixture(scope="module")
def pg():
    from paper_1705_02313_gb300 import build, pg as _pg
    build.build()
    return _pg


@pytest.fixture(scope="module")
def ctx(pg):
    c = pg.pg_ctx_create(0)
    yield c
    pg.pg_ctx_destroy(c)


@pytest.fixture(scope="module")
def game():
    g = gen.native_random_game(N, DMIN, DMAX, SEED)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    return g, gp


@pytest.fixture(scope="module")
def game_cv():
    g = gen.native_random_game(N, DMIN, DMAX, SEED, levels=4)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    return g, gp


def gpu_solve(pg, ctx, g, max_inner=0):
    """pg_load_csr from device arrays, pg_solve into device arrays; returns
    host copies, the status and the iteration counts."""
    import torch
    d = [torch.from_numpy(a).cuda() for a in g.arrays()]
    game = pg.pg_load_csr(ctx, g.n, g.m, *d)
    try:
        _, _, k = pg.pg_game_info(game)
        nlev = pg.pg_game_levels(game).size
        dev = dict(win=torch.empty(g.n, dtype=torch.uint8, device="cuda"),
                   sigma=torch.empty(g.n, dtype=torch.int32, device="cuda"),
                   tau=torch.empty(g.n, dtype=torch.int32, device="cuda"),
                   val_class=torch.empty(g.n, dtype=torch.int8, device="cuda"),
                   val_depth=torch.empty(g.n, dtype=torch.int32, device="cuda"),
                   val_rank=torch.empty(g.n, dtype=torch.int32, device="cuda"),
                   dummy_sigma=torch.empty(max(k, 1), dtype=torch.int8, device="cuda"))
        if nlev:
            dev["val_counts"] = torch.empty(g.n * nlev, dtype=torch.int32, device="cuda")
        try:
            major, inner = pg.pg_solve(ctx, game, max_inner=max_inner, **dev)
            rc = pg.PG_OK
        except pg.PgError as e:
            rc, major, inner = e.code, None, None
        used, iters = pg.pg_last_loop(game)
        torch.cuda.synchronize()
        out = {key: t.cpu().numpy() for key, t in dev.items()}
        out["dummy_sigma"] = out["dummy_sigma"][:k]
        if nlev:
            out["val_counts"] = out["val_counts"].reshape(g.n, nlev)
    finally:
        pg.pg_game_free(game)
    return rc, major, inner, used, iters, out


def assert_equal(got, want, keys, label):
    for key in keys:
        a, b = np.asarray(got[key]), np.asarray(want[key])
        if not np.array_equal(a, b):
            bad = np.nonzero(a != b)[0]
            raise AssertionError("%s: %s differs at %d vertices, first %s: got %s want %s" %
                                 (label, key, bad.size, bad[:5], a[bad[:5]], b[bad[:5]]))


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size_digests.json")
FINAL_KEYS = ["win", "sigma", "tau", "val_class", "val_depth", "val_rank", "dummy_sigma"]


def workload(name):
    if name == "random-10m":
        return gen.native_random_game(N, DMIN, DMAX, SEED)
    return gen.ladder_game(N, SEED)


@pytest.mark.parametrize("name", ["random-10m", "ladder-10m"])
def test_full_size_final_results_equal_oracle(pg, ctx, name):
    rec = json.load(open(GOLDEN))["workloads"][name]
    g = workload(name)
    h = hashlib.sha256()
    for a in g.arrays():
        h.update(np.ascontiguousarray(a).tobytes())
    assert h.hexdigest() == rec["input_sha256"], "the generator changed: rerun tests/golden/make_full_size_digests.py"
    rc, major, inner, used, iters, got = gpu_solve(pg, ctx, g)
    assert rc == pg.PG_OK and used and iters == inner
    bad = []
    for key in FINAL_KEYS:
        a, want = np.ascontiguousarray(got[key]), rec["arrays"][key]
        assert str(a.dtype) == want["dtype"] and a.size == want["size"], key
        idx = np.asarray(want["sample_index"], np.int64)
        assert a[idx].astype(np.int64).tolist() == want["sample_value"], key  # sampled values, element by element
        if hashlib.sha256(a.tobytes()).hexdigest() != want["sha256"]:
            bad.append(key)
    assert not bad, "%s: arrays differing from the oracle's full solve: %s" % (name, bad)
    assert (major, inner) == (rec["major"], rec["inner"])


def test_full_size_first_valuations(pg, ctx, game):
    g, gp = game
    rc, _, _, used, iters, got = gpu_solve(pg, ctx, g, max_inner=3)
    assert rc == pg.PG_ETIMEOUT and used and iters == 3
    r = o2.run(gp, max_inner=3, allow_timeout=True)
    assert r["status"] == o2.ETIMEOUT and r["inner"] == 3
    sigma, tau, dsig = profile_to_original(gp, r["strat"])
    assert_equal(got, dict(sigma=sigma, tau=tau, dummy_sigma=dsig), ["sigma", "tau", "dummy_sigma"], "profile")
    val = o2.valuate(gp, r["strat"])  # the valuation of the profile the cap returns
    want = o2.map_back(gp, dict(val, strat=r["strat"]))
    assert_equal(got, want, ["win", "val_class", "val_depth", "val_rank"], "valuation")


def test_full_size_solution_certified(pg, ctx, game):
    g, gp = game
    rc, major, inner, used, iters, got = gpu_solve(pg, ctx, g)
    assert rc == pg.PG_OK and used and iters == inner and major > 0
    cert.certify(gp, g.offsets, g.targets, got)
    assert 0 < int(got["win"].sum()) < g.n  # both players win somewhere


def test_full_size_count_vectors_first_valuations(pg, ctx, game_cv):
    g, gp = game_cv
    rc, _, _, used, iters, got = gpu_solve(pg, ctx, g, max_inner=3)
    assert rc == pg.PG_ETIMEOUT and used and iters == 3
    r = o3.run(gp, max_inner=3, allow_timeout=True)
    assert r["status"] == o3.ETIMEOUT and r["inner"] == 3
    sigma, tau, dsig = profile_to_original(gp, r["strat"])
    assert_equal(got, dict(sigma=sigma, tau=tau, dummy_sigma=dsig), ["sigma", "tau", "dummy_sigma"], "profile")
    val = o3.valuate(gp, r["strat"])
    want = o3.map_back(gp, dict(val, strat=r["strat"]))
    assert_equal(got, want, ["win", "val_class", "val_depth", "val_counts"], "valuation")
    assert (got["val_rank"] == -1).all()


def test_full_size_count_vectors_certified(pg, ctx, game_cv):
    g, gp = game_cv
    rc, major, inner, used, iters, got = gpu_solve(pg, ctx, g)
    assert rc == pg.PG_OK and used and iters == inner and major > 0
    cert.certify_counts(gp, g.offsets, g.targets, got)


@pytest.mark.parametrize("levels", [3, 4])
def test_count_vectors_beyond_2_24_ids(pg, ctx, levels):
    """20M-vertex random games with 3 and 4 priorities (4 and 5 levels with
    the dummies'): more than 2^24 ids after preprocessing, beyond fixed 25-bit
    digits; with 4 priorities the shape of the largest games of Table 1."""
    g = gen.native_random_game(20_000_000, DMIN, DMAX, 3, levels=levels)
    gp = o2.preprocess(g.n, g.offsets, g.targets, g.owner, g.pri)
    assert gp["n"] + 1 > (1 << 24) and gp["k"] > 0
    rc, _, _, used, iters, got = gpu_solve(pg, ctx, g, max_inner=3)
    assert rc == pg.PG_ETIMEOUT and used and iters == 3
    r = o3.run(gp, max_inner=3, allow_timeout=True)
    assert r["status"] == o3.ETIMEOUT and r["inner"] == 3
    sigma, tau, dsig = profile_to_original(gp, r["strat"])
    assert_equal(got, dict(sigma=sigma, tau=tau, dummy_sigma=dsig), ["sigma", "tau", "dummy_sigma"], "profile")
    val = o3.valuate(gp, r["strat"])
    want = o3.map_back(gp, dict(val, strat=r["strat"]))
    assert_equal(got, want, ["win", "val_class", "val_depth", "val_counts"], "valuation")
    assert got["val_counts"].shape == (g.n, levels + 1)
    rc, major, inner, used, iters, got = gpu_solve(pg, ctx, g)
    assert rc == pg.PG_OK and used and iters == inner and major > 0
    cert.certify_counts(gp, g.offsets, g.targets, got)
