"""bench.py's roofline arithmetic (host logic, no GPU): the algorithmic work
per launch of the panel and of the trailing update, checked against
element-by-element counts, and the rule that a stored DRAM-traffic capture is
used only for the kernel source it was taken on."""
import numpy as np
import pytest

import bench


def _panel_macs_brute(n, w):
    """Complex multiply-accumulates of all panel launches of width w on an n x n
    matrix, counted element by element: at column j of a panel [s0, s0+w)
    every row below j gets its multiplier (1) and its rank-1 update of the
    panel columns right of j."""
    total = 0
    for s0 in range(0, n, w):
        s1 = min(s0 + w, n)
        for j in range(s0, s1):
            for i in range(j + 1, n):
                total += 1                      # multiplier l_ij
                total += s1 - (j + 1)          # a_ic -= l_ij u_jc, c in (j, s1)
    return total


@pytest.mark.parametrize("n,w", [(70, 32), (64, 32), (33, 32), (40, 16)])
def test_panel_work_matches_element_count(n, w):
    steps, launches = 2, 2 * ((n + w - 1) // w)
    prof = {"panel": (10.0, launches)}
    method, nb = ("ozaki", 128) if w == 32 else ("4m", w)
    r = bench.panel_roofline(method, "dd", n, nb, steps, prof, el_ms=100.0)
    ops = _panel_macs_brute(n, w) * 4 * bench.I_REAL["dd"]
    assert r["ops_per_launch"] * launches / steps == pytest.approx(ops)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["achieved"] == pytest.approx(r["ops_per_launch"] / (10.0 / launches * 1e-3) / 1e12)
    assert r["share_of_step"] == pytest.approx(0.1)


def test_ozaki_update_flops_match_slice_pair_count():
    n, nb, steps = 300, 128, 1
    blocks = [(j0, min(nb, n - j0)) for j0 in range(0, n, nb)]
    launches = sum(1 for j0, jb in blocks if n - j0 - jb > 0)
    r = bench.roofline("ozaki", "dd", n, nb, steps, {"gemm": (5.0, launches)}, el_ms=50.0)
    S = bench.OZAKI_S["dd"]
    kept = sum(1 for p in range(S) for q in range(S) if p + q < S)   # slice pairs on or above the anti-diagonal
    flops = sum(kept * 2.0 * (n - j0 - jb) * 2 * (n - j0 - jb) * 2 * jb for j0, jb in blocks)
    assert r["flops_per_launch"] * launches == pytest.approx(flops)
    assert r["unit"] == "TFLOP/s" and r["bound"] == "tensor"


def test_plain_update_ops_match_mac_count():
    n, nb, steps = 200, 64, 1
    macs = 0
    for j0 in range(0, n, nb):
        jb = min(nb, n - j0)
        n2 = n - j0 - jb
        macs += int(np.int64(n2) * n2 * jb)
    launches = sum(1 for j0 in range(0, n, nb) if n - j0 - min(nb, n - j0) > 0)
    for method, per in (("4m", 4), ("3m", 3)):
        r = bench.roofline(method, "td", n, nb, steps, {"gemm": (3.0, launches)}, el_ms=30.0)
        assert r["ops_per_launch"] * launches == pytest.approx(macs * per * bench.I_REAL["td"])


def _sha(name):
    import hashlib
    import os
    with open(os.path.join(bench.ROOT, "paper_2403_16013_gb300", "csrc", name), "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()


def test_panel_traffic_only_for_the_captured_source(monkeypatch):
    n, steps = 4096, 1
    launches = n // 32
    prof = {"panel": (40.0, launches)}
    # a capture taken on the current source is used ...
    monkeypatch.setitem(bench.PANEL_TRAFFIC, "dd", dict(bench.PANEL_TRAFFIC["dd"], src_sha1=_sha("panel_coop.cuh")))
    r = bench.panel_roofline("ozaki", "dd", n, 128, steps, prof, el_ms=100.0)
    cap = bench.PANEL_TRAFFIC["dd"]
    rows = [n - s0 for s0 in range(0, n, 32)]
    assert r["traffic"] == pytest.approx(cap["bytes"] * np.mean(rows) / cap["m"])
    # another kernel source: no traffic
    monkeypatch.setitem(bench.PANEL_TRAFFIC, "dd", dict(cap, src_sha1="0" * 40))
    assert bench.panel_roofline("ozaki", "dd", n, 128, steps, prof, el_ms=100.0)["traffic"] is None
    # another precision or launch width: no traffic
    assert bench.panel_roofline("ozaki", "td", n, 128, steps, prof, el_ms=100.0)["traffic"] is None
    assert bench.panel_roofline("4m", "dd", n, 64, steps, prof, el_ms=100.0)["traffic"] is None


def test_trailing_traffic_only_for_the_captured_source(monkeypatch):
    n, nb, steps = 4096, 128, 1
    launches = n // nb - 1
    monkeypatch.setitem(bench.OZ_TRAFFIC, "dd", dict(bench.OZ_TRAFFIC["dd"], src_sha1=_sha("ozaki.cuh")))
    r = bench.roofline("ozaki", "dd", n, nb, steps, {"gemm": (27.8, launches)}, el_ms=111.6)
    cap = bench.OZ_TRAFFIC["dd"]
    n2s = [n - j0 - nb for j0 in range(0, n - nb, nb)]
    assert r["traffic"] == pytest.approx(cap["bytes"] * np.mean(np.square(n2s)) / cap["n2"] ** 2)
    monkeypatch.setitem(bench.OZ_TRAFFIC, "dd", dict(cap, src_sha1="0" * 40))
    assert bench.roofline("ozaki", "dd", n, nb, steps, {"gemm": (27.8, launches)}, el_ms=111.6)["traffic"] is None
