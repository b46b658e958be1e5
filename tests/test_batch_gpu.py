"""GPU parity of the batched persistent launch (flyte_batch_prepare / flyte_batch_launch).

Every job of a mixed batch is checked against the oracle with the bound of
its single-job entry point: unpack and axpy bit-exact (NaN by class), dot
within 4n 2^-53 sum|xy|, gemv within 4(len+2) 2^-53 (|alpha| sum|Ax| + |beta y|).
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from paper_1601_07789_gb300 import flyte, inputs
from tests.gpu_util import sync

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


class Batch:
    """Host data, device buffers and jobs for a list of specs (inputs.batch_specs)."""

    def __init__(self, specs, seed=1, offset=0):
        g = np.random.default_rng(seed)
        self.specs = specs
        self.host = []
        self.dev = []
        self.jobs = []
        self.naxpy = 0
        for s in specs:
            op, k, base, n, m = s["op"], s["k"], s["base"], s["n"], s["m"]
            dt = np.float32 if base == 0 else np.float64
            fx = (k, base)
            h = {}
            d = {}
            if op in (0, 1, 2):
                h["x"] = oracle.pack(g.standard_normal(n).astype(dt), base, k)
                d["x"] = self._dev(h["x"], offset)
            if op == 0:
                d["y"] = torch.zeros(n, dtype=torch.float32 if base == 0 else torch.float64, device="cuda")
                job = flyte.job(flyte.JOB_UNPACK, fx, n, d["x"], d["y"])
            elif op == 1:
                h["y"] = oracle.pack(g.standard_normal(n).astype(dt), base, k)
                d["y"] = self._dev(h["y"], offset)
                d["r"] = torch.full((), np.nan, dtype=torch.float64, device="cuda")
                job = flyte.job(flyte.JOB_DOT, fx, n, d["x"], d["y"], fy=fx, result=d["r"])
            elif op == 2:
                h["y"] = oracle.pack(g.standard_normal(n).astype(dt), base, k)
                d["y"] = self._dev(h["y"], offset)
                # every other axpy job takes a binary32 alpha (the exact binary32 path for double-based
                # k <= 4) and the rounding mode cycles through the four
                self.naxpy += 1
                a = g.uniform(-2, 2)
                h["alpha"] = float(np.float32(a)) if self.naxpy % 2 else float(a)
                h["mode"] = self.naxpy % 4
                job = flyte.job(flyte.JOB_AXPY, fx, n, d["x"], d["y"], fy=fx, alpha=h["alpha"], mode=h["mode"])
            else:
                h["A"] = oracle.pack(g.standard_normal(m * n).astype(dt), base, k)
                lx, ly = (n, m) if op == 3 else (m, n)
                h["xv"] = g.standard_normal(lx)
                h["y0"] = g.standard_normal(ly)
                h["alpha"], h["beta"] = 1.5, -0.5
                d["A"] = self._dev(h["A"], offset)
                d["xv"] = torch.from_numpy(h["xv"]).cuda()
                d["y"] = torch.from_numpy(h["y0"].copy()).cuda()
                job = flyte.job(flyte.JOB_GEMV_N if op == 3 else flyte.JOB_GEMV_T, fx, n, d["A"], d["y"], m=m,
                                xv=d["xv"], alpha=1.5, beta=-0.5)
            self.host.append(h)
            self.dev.append(d)
            self.jobs.append(job)

    @staticmethod
    def _dev(a, offset):
        buf = torch.zeros(a.size + offset + 16, dtype=torch.uint8, device="cuda")
        buf[offset:offset + a.size] = torch.from_numpy(a).cuda()
        return buf[offset:]

    def check(self, skip_axpy=False, gemv_sample=None):
        """gemv_sample: check only that many output entries per gemv job (rows of A for 'N', columns
        for 'T', seeded, always including the first and last), against the oracle on those rows or
        columns of A alone."""
        for s, h, d in zip(self.specs, self.host, self.dev):
            op, k, base, n, m = s["op"], s["k"], s["base"], s["n"], s["m"]
            if op == 0:
                got = d["y"].cpu().numpy()
                want = oracle.unpack(h["x"], base, k).view(np.float32 if base == 0 else np.float64)
                assert np.array_equal(got.view(want.dtype).view(np.uint8), want.view(np.uint8)), s
            elif op == 1:
                if n == 0:
                    assert float(d["r"].item()) == 0.0
                    continue
                ref, _, absum = oracle.dot(n, h["x"], (base, k), 1, h["y"], (base, k), 1)
                got = float(d["r"].item())
                assert abs(got - ref) <= 4 * n * EPS * absum + 2 * EPS * abs(ref), s
            elif op == 2 and not skip_axpy:
                got = d["y"][: n * k].cpu().numpy()
                want = oracle.axpy(n, h["alpha"], h["x"], (base, k), 1, h["y"], (base, k), 1, h["mode"])
                assert np.array_equal(got, want), s
            elif op >= 3:
                trans = "N" if op == 3 else "T"
                got = d["y"].cpu().numpy()
                L = n if op == 3 else m
                ly = m if op == 3 else n
                if gemv_sample is None or gemv_sample >= ly:
                    idx = np.arange(ly)
                    ref, absum = oracle.gemv(trans, m, n, 1.5, h["A"], (base, k), n, h["xv"], 1, -0.5, h["y0"], 1)
                else:
                    g = np.random.default_rng(ly * 7 + L)
                    idx = np.unique(np.concatenate([[0, ly - 1], g.integers(0, ly, gemv_sample)]))
                    codes = h["A"].reshape(m, n, k)
                    sub = np.ascontiguousarray(codes[idx] if op == 3 else codes[:, idx]).reshape(-1)
                    mm, nn = (idx.size, n) if op == 3 else (m, idx.size)
                    ref, absum = oracle.gemv(trans, mm, nn, 1.5, sub, (base, k), nn, h["xv"], 1, -0.5,
                                             h["y0"][idx], 1)
                    got = got[idx]
                bound = 4 * (L + 2) * EPS * (1.5 * absum + 0.5 * np.abs(h["y0"][idx])) + 2 * EPS * np.abs(ref)
                assert np.all(np.abs(got - ref) <= bound), s


SPECS = inputs.batch_specs(160, seed=5, len_range=(1, 2e5), side_range=(1, 700))


def test_batch_mixed_jobs():
    b = Batch(SPECS)
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check()


def test_batch_replay_and_graph():
    """Launching again (counters reset by the kernel) and replaying a captured CUDA graph give the same
    results; axpy jobs are left out (they update in place)."""
    specs = [s for s in SPECS if s["op"] != 2][:80]
    b = Batch(specs, seed=2)
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check()
    first = [d["y"].clone() if s["op"] != 1 else d["r"].clone() for s, d in zip(specs, b.dev)]
    stream = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        flyte.batch_launch(ws, stream=stream)
    for _ in range(3):
        for i, s in enumerate(specs):
            if s["op"] >= 3:
                b.dev[i]["y"].copy_(torch.from_numpy(b.host[i]["y0"]))
        graph.replay()
        sync()
        again = [d["y"] if s["op"] != 1 else d["r"] for s, d in zip(specs, b.dev)]
        for a, c in zip(first, again):
            assert torch.equal(a, c)


def test_batch_misaligned_and_edges():
    specs = [{"op": op, "k": k, "base": base, "n": n, "m": m}
             for (op, k, base, n, m) in [(0, 3, 1, 1001, 0), (1, 5, 1, 999, 0), (2, 7, 1, 1003, 0), (3, 3, 1, 77, 65),
                                         (4, 6, 1, 63, 130), (1, 2, 0, 4097, 0), (0, 3, 0, 7, 0), (1, 4, 1, 0, 0),
                                         (3, 2, 1, 5, 0), (4, 5, 1, 3, 1)]]
    b = Batch(specs, seed=3, offset=1)
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check()
    with pytest.raises(flyte.FlyteError):
        flyte.batch_prepare([flyte.job(flyte.JOB_GEMV_N, (4, 1), 5000, b.dev[0]["x"], b.dev[0]["x"], m=4,
                                       xv=b.dev[0]["x"])])   # gemv side above the batch limit


# 'T' jobs narrower than 1024 columns cut each tile's rows among G thread groups (G = 16, 8, 4, 2, 1
# here, one with a ragged last group) and 'N' jobs share an x split once per launch across many row
# tiles (one on the double-word tree, one on the binary64 row sums): against the oracle, and a second
# launch gives the same bits.
NARROW = [{"op": 4, "k": k, "base": 1, "n": n, "m": 4096}
          for k, n in ((3, 64), (5, 66), (4, 100), (6, 200), (2, 500), (7, 1000))] + [
    {"op": 3, "k": 4, "base": 1, "n": 1500, "m": 3000},
    {"op": 3, "k": 5, "base": 1, "n": 600, "m": 2000},
]


def test_batch_narrow_t_groups_and_split_x():
    b = Batch(NARROW, seed=31)
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check(gemv_sample=300)
    first = [d["y"].clone() for d in b.dev]
    for i, s in enumerate(NARROW):
        b.dev[i]["y"].copy_(torch.from_numpy(b.host[i]["y0"]))
    flyte.batch_launch(ws)
    sync()
    for a, d in zip(first, b.dev):
        assert torch.equal(a, d["y"])


# The batched workload's own size distribution (vector lengths log-uniform in 10^3..10^6, gemv sides
# log-uniform in 64..4096), plus jobs that reach the paths only large sides take: 'T' jobs several
# 1024-column blocks wide and gemv jobs whose x (staged in shared memory) has 4096 entries.
CONFIG5 = inputs.batch_specs(40, seed=11, len_range=(1e3, 1e6), side_range=(64, 4096)) + [
    {"op": 4, "k": 5, "base": 1, "n": 4096, "m": 1500},     # 'T', 4 column blocks, x of 1500
    {"op": 4, "k": 3, "base": 0, "n": 3001, "m": 4096},     # 'T', 3 blocks + ragged, x of 4096
    {"op": 3, "k": 6, "base": 1, "n": 4096, "m": 700},      # 'N', x of 4096
    {"op": 3, "k": 2, "base": 1, "n": 4095, "m": 4096},     # 'N', ragged rows, x of 4095
    {"op": 4, "k": 7, "base": 1, "n": 2049, "m": 4096},     # 'T', 3 blocks, one of a single column
]


def _config5_run():
    b = Batch(CONFIG5, seed=12)
    assert any(s["op"] == 4 and s["n"] > 1024 for s in CONFIG5)
    assert max(s["n"] if s["op"] == 3 else s["m"] for s in CONFIG5 if s["op"] >= 3) == 4096
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check(gemv_sample=200)


def test_batch_config5_sizes_default_tiles():
    """Runs before any autotuning in this file: the built-in tile table."""
    _config5_run()


def test_batch_autotune_then_run():
    flyte.batch_autotune()
    b = Batch(SPECS[:60], seed=4)
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check()


def test_batch_autotune_on_the_job_mix():
    """flyte_batch_autotune_jobs times candidates on the caller's own batch; afterwards the table holds
    candidate sizes, the persistent launch at least one block per SM, and the batch stays exact."""
    specs = [s for s in inputs.batch_specs(48, seed=21, len_range=(1e3, 3e5), side_range=(64, 1500))]
    tune = Batch(specs, seed=22)
    flyte.batch_autotune_jobs(tune.jobs)
    assert flyte.batch_resident_blocks() >= 1
    for sp in specs:
        f = (sp["k"], sp["base"])
        t = flyte.batch_tile_size(sp["op"], f)
        allowed = {0: {16384, 32768, 65536, 131072, 262144}, 1: {16384, 32768, 65536, 131072, 262144},
                   2: {16384, 32768, 65536, 131072, 262144}, 3: {4, 8, 16, 32}, 4: {128, 256, 512}}[sp["op"]]
        assert t in allowed, (sp, t)
    assert flyte.batch_tile_size(9, (4, 1)) == -1
    b = Batch(specs, seed=23)                      # fresh data: the tuning runs changed the axpy outputs
    ws = flyte.batch_prepare(b.jobs)
    flyte.batch_launch(ws)
    sync()
    b.check()


def test_batch_config5_sizes_autotuned_tiles():
    """The same jobs after flyte_batch_autotune has filled the tile table."""
    flyte.batch_autotune()
    _config5_run()
