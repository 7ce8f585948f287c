"""Host-side pieces of bench.py that need no GPU: the per-kernel DRAM traffic recorded with
ncu is reported only for the kernel source it was taken from; the whole-job throughput and
the roofline arithmetic."""
import bench


def test_recorded_traffic_follows_the_kernel_source(monkeypatch, tmp_path):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic_sweep.txt").write_text(
        "# comment\nkernel_source_sha256 " + "a" * 64 + "\nenum_kernel 968448\nrows_kernel 2000 500\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "a" * 64)
    got = bench.recorded_traffic("sweep")
    assert got == {"enum_kernel": (968448, None), "rows_kernel": (2000, 500)}
    # a capture of a smaller case scales with the full launch's units; a full-size one does not
    assert bench.scaled_traffic(got["rows_kernel"], 5000) == 20000
    assert bench.scaled_traffic(got["enum_kernel"], 123) == 968448
    assert bench.scaled_traffic(None, 1) is None
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 64)
    assert bench.recorded_traffic("sweep") == {}
    assert bench.recorded_traffic("no_such_workload") == {}


def test_kernel_rooflines_pick_the_largest_share():
    prof = {"ms_enum": 0.1, "ms_rows": 0.4, "ms_count": 0.2, "ms_model": 0.02, "ms_rank": 0.01, "ms_total": 0.73,
            "block_addresses": 1_000_000, "row_reds": 40_000_000, "bitmap_bytes": 4_000_000_000,
            "count_bytes": 1_000_000_000, "passes": 1}
    peaks = {"int_ops_per_s": 3.0e13, "l2_red_per_s": 2.0e11}
    r = bench.kernel_rooflines([prof, prof, prof], peaks)
    assert r["kernel"] == "rows_kernel"
    assert abs(r["achieved"] - 40e6 / 0.4e-3 / 1e9) < 1e-9          # G red.or / s
    assert abs(r["frac"] - (40e6 / 0.4e-3) / 2.0e11) < 1e-12
    c = r["kernels"]["count_kernel"]
    assert abs(c["achieved"] - 1e9 / 0.2e-3 / 1e9) < 1e-9          # GB / s
    assert r["traffic"] is None                                     # no workload given


def test_job_throughput_counts_all_ranks():
    assert bench.job_throughput(755, 1, 1.0) == 755_000.0
    assert bench.job_throughput(755, 4, 2.0) == 4 * 755 / 2e-3


def test_rows_roofline_uses_the_run_pattern_peak_when_measured():
    prof = {"ms_enum": 0.1, "ms_rows": 0.4, "ms_count": 0.2, "ms_model": 0.02, "ms_rank": 0.01, "ms_total": 0.73,
            "block_addresses": 1, "row_reds": 40_000_000, "bitmap_bytes": 1, "count_bytes": 1, "passes": 1}
    peaks = {"int_ops_per_s": 3.0e13, "l2_red_per_s": 2.0e11, "l2_red64_run_per_s": 4.0e11}
    r = bench.kernel_rooflines([prof], peaks)["kernels"]["rows_kernel"]
    assert abs(r["frac"] - (40e6 / 0.4e-3) / 4.0e11) < 1e-12 and r["peak_random_32bit"] == 200.0


def test_clock_summary():
    lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.summarize_clocks(lines)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert bench.summarize_clocks([]) is None


class _FakeServer:
    """Serves requests one after another, `service` seconds each (newest first when `lifo`,
    as a server that runs whole steps may finish later requests first); poll waits up to its
    timeout for a request that is not done, as ws_server_poll does."""

    WS_EAGAIN = -3

    def __init__(self, service=20e-6, lifo=False, n=0):
        import threading
        import time
        self.service, self.lifo, self.n_all = service, lifo, n
        self.due, self.n, self.free_at, self.mu = {}, 0, 0.0, threading.Lock()
        self.t0 = time.perf_counter()

    def submit(self, arrays=None):
        import time
        with self.mu:
            self.n += 1
            if self.lifo:   # all submitted at once: request i is served (n_all - i)-th
                self.due[self.n] = self.t0 + (self.n_all - self.n + 1) * self.service
            else:
                self.free_at = max(self.free_at, time.perf_counter()) + self.service
                self.due[self.n] = self.free_at
            return self.n

    def poll(self, rid, timeout_us=0):
        import time
        with self.mu:
            due = self.due[rid]
        now = time.perf_counter()
        if now < due:
            if timeout_us <= 0 or now + timeout_us * 1e-6 < due:
                time.sleep(timeout_us * 1e-6)
                return self.WS_EAGAIN, None, None
            time.sleep(due - now)
        with self.mu:
            del self.due[rid]
        return 0, [0] * 10, None


def test_served_requests_are_collected_as_they_finish():
    """The serving harness (submitter and poller threads) against a server stand-in: every
    request comes back once, with its candidates, whether the requests finish in submission
    order or newest first, in about the time the stand-in takes to serve them."""
    class B:
        WS_EAGAIN = _FakeServer.WS_EAGAIN
        WsError = RuntimeError
    n = 5000
    r = bench.serve_stream(B, _FakeServer(), [None] * n, [None] * n, [0.0] * n)
    assert r["ok"] == n and r["configs"] == 10 * n
    assert r["seconds"] < 0.5, r
    # newest first: the oldest requests finish last
    r = bench.serve_stream(B, _FakeServer(lifo=True, n=n), [None] * n, [None] * n, [0.0] * n)
    assert r["ok"] == n and r["p50_ms"] < 250.0, r
    # a paced stream below the service rate: every request back soon after its arrival
    m = 200
    r = bench.serve_stream(B, _FakeServer(), [None] * m, [None] * m, [i * 1e-3 for i in range(m)])
    assert r["ok"] == m and r["p50_ms"] < 10.0, r
