"""Host-side logic of the package on the CPU: the packed tile layout shared
with the oracle, identity padding for ragged sizes, the tile autotuner's
choice rule, the serving requests and their device footprint."""
import json

import numpy as np
import pytest
import torch

import synth
import paper_1304_0878_b300 as b3t
from paper_1304_0878_b300 import tiles as dt, batch as bt, tune, serve as sv
from oracle import cholesky as och


@pytest.mark.parametrize("N,b", [(256, 64), (384, 128), (512, 512)])
def test_tile_layout_matches_the_oracle(N, b):
    # the device helpers and the oracle pack the lower tiles identically:
    # tile (i, j) at j*T - j(j-1)/2 + (i - j), each tile column-major
    A = synth.spd_host(N, seed=N, shift=1.0)
    t = dt.to_tiles(torch.from_numpy(A), b).numpy()
    assert np.array_equal(t, och.to_tiles(A, b))
    assert np.array_equal(dt.pack_lower(torch.from_numpy(A), b).numpy(), t)
    T = N // b
    for i in range(T):
        for j in range(i + 1):
            assert dt.tile_index(i, j, T) == och.tile_index(i, j, T)
            assert np.array_equal(t[dt.tile_index(i, j, T)], A[i * b:(i + 1) * b, j * b:(j + 1) * b].T)
    back = dt.from_tiles(torch.from_numpy(t), N, b).numpy()
    L = np.zeros_like(A)
    for i in range(T):
        for j in range(i + 1):
            L[i * b:(i + 1) * b, j * b:(j + 1) * b] = A[i * b:(i + 1) * b, j * b:(j + 1) * b]
    assert np.array_equal(back, L)


def test_tile_ptrs_step_by_tile():
    t = torch.zeros((6, 4, 4), dtype=torch.float64)
    p = dt.tile_ptrs(t)
    assert p[0] == t.data_ptr() and all(q - r == 4 * 4 * 8 for r, q in zip(p, p[1:]))


@pytest.mark.parametrize("N,b", [(77, 64), (300, 128), (513, 256), (512, 128)])
def test_identity_padding(N, b):
    # a ragged size is padded to diag(A, I); its Cholesky factor is diag(L, I)
    A = torch.from_numpy(synth.spd_host(N, seed=3, shift=1.0))
    t, Np = bt.padded_tiles(A, b)
    assert Np == dt.pad_size(N, b) and Np % b == 0 and Np - N < b
    C = dt.from_tiles(t, Np, b).numpy()
    assert np.array_equal(np.tril(C[:N, :N]), np.tril(A.numpy()))
    assert np.array_equal(C[N:, N:], np.eye(Np - N))
    assert np.all(C[N:, :N] == 0)
    # the oracle factors the padded matrix to diag(L, I)
    Cs = np.tril(C) + np.tril(C, -1).T
    L, info = och.dense_potrf(Cs)
    assert info == 0
    L = np.tril(L)
    assert np.allclose(L[N:, N:], np.eye(Np - N)) and np.all(L[N:, :N] == 0)


def test_tile_choice_rule(tmp_path):
    table = {"fp64": {"256": {"best": 64}, "1024": {"best": 128}, "8192": {"best": 512}},
             "bf16": {"1024": {"best": 128}, "8192": {"best": 256}}}
    path = tmp_path / "table.json"
    path.write_text(json.dumps(table))
    try:
        tune.load(str(path))
        assert tune.choose_tile(1024, "fp64") == 128
        assert tune.choose_tile(900, "fp64") == 128          # nearest tuned size in log scale
        assert tune.choose_tile(300, "fp64") == 64
        assert tune.choose_tile(8192, "fp64") == 512
        assert tune.choose_tile(5000, "fp64") == 512          # log-nearest to 8192
        assert tune.choose_tile(200, "fp64") == 64
        assert tune.choose_tile(100, "bf16") == 128           # mixed tiles are at least 128
        assert tune.choose_tile(6000, "bf16") == 256
        # no more than one mostly padded tile: b halves while b >= 2N (down to 64)
        table["fp64"]["256"]["best"] = 512
        path.write_text(json.dumps(table))
        tune.load(str(path))
        assert tune.choose_tile(100, "fp64") == 128 and tune.choose_tile(256, "fp64") == 256
        # no measurements for a precision: the rule of thumb
        assert tune.choose_tile(3000, "e4m3") == tune.default_tile(3000, "e4m3") == 256
    finally:
        tune.load()


def test_committed_tile_table_is_complete():
    tab = tune.load()
    for prec in ("fp64", "bf16"):
        for n in tune.SIZES:
            row = tab[prec][str(n)]
            ms = {int(k): v for k, v in row["ms"].items()}
            assert row["best"] == min(ms, key=ms.get)
            assert set(ms) <= set(tune.TILES[prec])


def test_serving_requests():
    # the same requests at every rate (arrival gaps scale with 1/rate), sizes
    # log-uniform in range, tiles from the tuner, footprint from the layout
    a = sv.make_requests(64, 2000.0, seed=5)
    c = sv.make_requests(64, 20.0, seed=5)
    assert [(r.N, r.nrhs, r.seed) for r in a] == [(r.N, r.nrhs, r.seed) for r in c]
    ta = np.array([r.arrival for r in a])
    tc = np.array([r.arrival for r in c])
    assert np.all(np.diff(ta) > 0) and np.allclose(tc, ta * 100.0, rtol=1e-12)
    for r in a:
        assert 256 <= r.N <= 8192 and 1 <= r.nrhs <= 32
        assert r.b == tune.choose_tile(r.N, "fp64") and r.Np == dt.pad_size(r.N, r.b) and r.T * r.b == r.Np
        assert r.bytes == sv.footprint(r.Np, r.nrhs, r.b, "fp64")
    f = [r for r in sv.make_requests(8, 100.0, seed=5, prec="bf16", tile=256)]
    assert all(r.b == 256 for r in f)


def test_serving_stream_prefix_is_stable():
    # the first k requests of the stream do not depend on how many are drawn
    a = synth.serve_requests(2000)
    b = synth.serve_requests(256)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x)[:256], np.asarray(y))


def test_serving_requests_cycle_distinct_sources():
    # n requests over P input sources: request i keeps the i-th arrival of the
    # stream and takes size, right-hand sides and seed of request i mod P
    full = sv.make_requests(40, 2000.0, seed=5)
    cyc = sv.make_requests(40, 2000.0, seed=5, distinct=8)
    assert [r.arrival for r in cyc] == [r.arrival for r in full]
    for i, r in enumerate(cyc):
        s = full[i % 8]
        assert (r.src, r.N, r.nrhs, r.seed, r.b, r.bytes) == (i % 8, s.N, s.nrhs, s.seed, s.b, s.bytes)
    assert [r.src for r in full] == list(range(40))


def test_serving_timeline_bins():
    # samples: (t, queue, in flight, arrived, admitted, completed), counts
    # cumulative; bins report increments and the largest queue in the bin
    samples = [(0.1, 3, 1, 4, 1, 0), (0.4, 5, 2, 8, 3, 1), (0.6, 1, 2, 9, 7, 5), (1.0, 0, 0, 9, 9, 9)]
    tl = sv._timeline(samples, 1.0, bins=2)
    assert tl == [{"t_s": 0.5, "arrived": 8, "admitted": 3, "completed": 1, "max_queue": 5, "in_flight": 2},
                  {"t_s": 1.0, "arrived": 1, "admitted": 6, "completed": 8, "max_queue": 1, "in_flight": 0}]


def test_serve_oracle_helper_solves_the_padded_system():
    # the test helper that checks served solutions: packed tiles of diag(A, I)
    # and right-hand-side parts in, the oracle's X with A X = B out
    import serve_oracle
    from oracle import cholesky as och
    N, b, nrhs = 200, 64, 3
    Np = dt.pad_size(N, b)
    A = np.eye(Np)
    A[:N, :N] = synth.spd_host(N, seed=3, shift=1.0)
    Bm = np.zeros((Np, nrhs))
    Bm[:N] = synth.rhs(N, nrhs, seed=4)
    parts = np.ascontiguousarray(Bm.reshape(Np // b, b, nrhs).transpose(0, 2, 1))
    assert np.array_equal(serve_oracle.dense_rhs(parts), Bm)
    X, A2, B2 = serve_oracle.solve((och.to_tiles(A, b), parts, Np, b))
    assert np.array_equal(A2, A) and np.array_equal(B2, Bm)
    assert np.max(np.abs(A @ X - Bm)) <= 1e-12 * np.max(np.abs(Bm))
    assert np.all(X[N:] == 0.0)


def test_footprint_counts_every_buffer():
    # fp64: A + factor tiles; mixed: A (FP64), W (binary32), L (FP64), Q
    # (one byte per element for E4M3, two for bf16); two block vectors; the
    # refinement work area; 4 KiB of slack
    Np, nrhs, b = 1024, 8, 256
    T = Np // b
    nt = T * (T + 1) // 2 * b * b
    base = 2 * T * b * nrhs * 8 + b3t.ir_work_elems(T, b, nrhs) * 8 + 4096
    assert sv.footprint(Np, nrhs, b, "fp64") == nt * 16 + base
    assert sv.footprint(Np, nrhs, b, "bf16") == nt * 22 + base
    assert sv.footprint(Np, nrhs, b, "e4m3") == nt * 21 + base
    assert sv.footprint(2 * Np, nrhs, b, "fp64") > 3 * sv.footprint(Np, nrhs, b, "fp64")


def test_trace_summary():
    # critical path = longest chain of task spans along the edges; busy
    # fraction = item time over CTAs x makespan; a late successor is counted
    from paper_1304_0878_b300 import trace
    rec = np.dtype([("task", np.int32), ("item", np.int32), ("sm", np.int32), ("kind", np.int32),
                    ("t_start_ns", np.uint64), ("t_end_ns", np.uint64)])
    tr = np.zeros(5, dtype=rec)
    tr["task"] = [0, 1, 2, 2, 3]
    tr["kind"] = [b3t.POTRF, b3t.TRSM, b3t.GEMM, b3t.GEMM, b3t.SYRK]
    tr["t_start_ns"] = [0, 1000, 1000, 1500, 4000]
    tr["t_end_ns"] = [1000, 2000, 3000, 3500, 5000]
    ed = [(0, 1), (0, 2), (1, 3), (2, 3)]
    s = trace.summary(tr, 4, ed, 2)
    assert s["critical_path_ms"] == 4500 / 1e6 and s["makespan_ms"] == 5000 / 1e6
    assert s["cta_busy_frac"] == 0.7 and s["edges_violated"] == 0
    assert s["kinds"]["GEMM"]["items"] == 2 and s["kinds"]["GEMM"]["cta_time_share"] == 4000 / 7000
    assert set(s["kinds"]) == {"POTRF", "TRSM", "GEMM", "SYRK"}
    # the path is POTRF -> GEMM (task 2, span 1000..3500) -> SYRK; SYRK waited 500 ns
    assert s["critical_path_tasks"] == 3
    assert s["critical_path_ms_by_kind"] == {"POTRF": 1000 / 1e6, "GEMM": 2500 / 1e6, "SYRK": 1000 / 1e6}
    assert s["critical_path_wait_ms"] == 500 / 1e6
    tr["t_start_ns"][4] = 3200          # task 3 starts before task 2 ends
    assert trace.summary(tr, 4, ed, 2)["edges_violated"] == 1
    assert trace.summary(tr[:1], 1, [], 1)["critical_path_ms"] == 1000 / 1e6    # no edges


def test_reference_arm_line_on_the_host():
    # the reference arm (the oracle, as it stands, on a bounded sample)
    # prints one JSON line with the same metric and workload config as the
    # device arm, its CPU baseline and a zero-copy e2e entry
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.check_output([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                                   "--n", "1024", "--b", "256", "--steps", "1", "--warmup", "0",
                                   "--cpu-seconds", "0.5"], cwd=root, env=env, text=True, timeout=300)
    line = json.loads(out.strip().splitlines()[-1])
    import bench
    assert line["impl"] == "reference" and line["metric"] == "cholesky_fp64_tflops"
    assert line["unit"] == "TFLOP/s" and line["higher_is_better"] is True and line["value"] > 0
    cfg = bench.workload_config(1024, 256)
    assert {k: line["config"][k] for k in cfg} == cfg
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"] == {"value": line["value"], "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_bench_host_checks_match_dense_definitions():
    # the benchmark's per-result error: rows of the symmetric A gathered from
    # packed lower tiles, the exact infinity norm, and the sampled normwise
    # backward error, against the same quantities on the dense matrix
    import bench
    from oracle import ir as oir
    N, b, nrhs = 256, 64, 3
    A = synth.spd_host(N, seed=9, shift=1.0)
    tl = och.to_tiles(A, b)
    for i in range(0, N, 17):
        assert np.array_equal(bench.host_sym_row(tl, i, N, b), A[i])
    assert bench.host_anorm(tl, N, b) == pytest.approx(np.max(np.sum(np.abs(A), axis=1)), rel=1e-14)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((N, nrhs))
    Bh = A @ X + 1e-9 * rng.standard_normal((N, nrhs))
    full = oir.backward_error(A, X, Bh)
    got = bench.sampled_host_eta(tl, bench.host_anorm(tl, N, b), X, Bh, N, b, nsamp=N * 4)
    assert got <= full * (1 + 1e-12) and got >= 0.5 * full


def test_bench_summary_keeps_the_headline_figures():
    import bench
    line = {"value": 1.2, "roofline": {"frac": 0.98}, "e2e": {"value": 1.1},
            "secondary": {"vector_chains": {"ms": 2.6, "hbm_frac": 0.99},
                          "vector_chains_item_chains": {"ms": 0.4, "floor_ms": 0.331, "hbm_frac": 0.83},
                          "empty_dags": {"chains": {"tasks_per_s": 4.5e6}},
                          "cholesky_small": {"ms": 5.0},
                          "time_to_solution": {"fp64": {"ms": 10000.0},
                                               "bf16": {"ms": 600.0, "factor_ms": 400.0, "speedup_vs_fp64": 16.0,
                                                        "eta": 1e-14, "host_sampled_eta": 2e-14,
                                                        "iterations": 5}},
                          "serving": {"fp64": {"continuous": {"requests": 2000, "p50_ms": 1.0, "p99_ms": 2.0,
                                                              "solves_per_s": 80.0, "max_queue": 5},
                                               "plain": {"requests": 256, "solves_per_s": 40.0,
                                                         "p99_ms": 9.0}}}},
            "cpu_baseline": {"value": 1e-3, "library": {"cores": 16, "cholesky_n1024": {"ms": 3.0}}}}
    sm = bench.summarise(line)
    assert sm["cholesky_fp64_tflops"] == 1.2 and sm["vector_chains"]["hbm_frac"] == 0.99
    assert sm["vector_chains_item_chains"] == {"ms": 0.4, "floor_ms": 0.331, "hbm_frac": 0.83}
    assert sm["tasks_per_s"]["chains"] == 4.5e6 and sm["cholesky_small_ms"] == 5.0
    assert sm["time_to_solution"]["bf16"]["host_sampled_eta"] == 2e-14
    assert sm["serving"]["fp64"]["requests"] == 2000 and sm["serving"]["fp64"]["plain_requests"] == 256
    assert sm["cpu"]["scipy_cores"] == 16 and sm["cpu"]["scipy_cholesky_n32768_tflops"] is None
