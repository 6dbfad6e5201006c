"""Host logic of the serving benchmark's measured one-at-a-time comparator
(bench._sequential_server), on the CPU with a stand-in library whose solve takes a fixed
time: requests are served first come first served, a request that arrives while another
is being solved waits for it, and latency runs from arrival to completion."""
import os
import sys
import time
import types

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

SOLVE_S = 0.05


class _Info:
    iters = 7
    rel_res_true = 5e-7


class _Handle:
    made = []

    def __init__(self, dim, n, theta_beta, k=None, precision=None, restart=None, maxit=None):
        _Handle.made.append((dim, n, precision))

    def solve_host(self, b, x, tol):
        time.sleep(SOLVE_S)
        return _Info()

    def close(self):
        pass


def _request(arrival, dim, n):
    work = types.SimpleNamespace(dim=dim, n=n, k=20.0, theta_beta=0.3, restart=40, tol=1e-6)
    return types.SimpleNamespace(arrival=arrival, work=work)


def test_sequential_server_is_first_come_first_served():
    stream = [_request(0.0, 2, 31), _request(0.0, 2, 31), _request(0.0, 3, 15), _request(0.5, 2, 31)]
    shapes = {(2, 31), (3, 15)}
    srcs = {sh: [torch.zeros(4, dtype=torch.complex128)] * 2 for sh in shapes}
    xbuf = {sh: [torch.zeros(4, dtype=torch.complex128)] * 2 for sh in shapes}
    _Handle.made.clear()
    out = bench._sequential_server(types.SimpleNamespace(Handle=_Handle), stream, srcs, xbuf, "c128")
    # one untimed warm-up request per shape, then a fresh handle per request
    assert len(_Handle.made) == len(shapes) + len(stream)
    assert all(p == "c128" for _, _, p in _Handle.made)
    assert out["iters_total"] == 7 * len(stream) and out["max_rel_res_true"] == 5e-7
    # three requests arrive together and finish one solve apart (latencies 1, 2, 3 solve
    # times); the fourth arrives after the queue has drained and waits for nobody (1):
    # median 1.5 solve times, 99th percentile about 3
    assert 1.5 * SOLVE_S - 0.01 <= out["p50_s"] < 1.5 * SOLVE_S + 0.05
    assert 2.9 * SOLVE_S <= out["p99_s"] < 3 * SOLVE_S + 0.1
    assert 0 < out["solves_per_s"] <= len(stream) / (0.5 + SOLVE_S)
