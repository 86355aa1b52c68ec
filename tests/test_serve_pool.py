"""The serving engine's device-pool allocator (host C++, no GPU needed).

The allocator in ``csrc/velo_pool.hpp`` is compiled into a small driver and
run against a byte-map model of first fit: each allocation must return the
lowest offset where n free bytes start a free run, releases must make the
bytes free again, the free list must equal the maximal free runs of the map
(so adjacent free ranges are always merged), and used / peak / largest-free
must match the map.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1912_09161_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    exe = str(tmp_path_factory.mktemp("pool") / "pool_check")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, os.path.join(ROOT, "tests", "native", "pool_check.cpp"),
                    "-o", exe], check=True)
    return exe


def _runs(free: np.ndarray):
    """Maximal runs of free bytes as (offset, size)."""
    out, i, n = [], 0, len(free)
    while i < n:
        if free[i]:
            j = i
            while j < n and free[j]:
                j += 1
            out.append((i, j - i))
            i = j
        else:
            i += 1
    return out


def _first_fit(free: np.ndarray, k: int):
    for off, size in _runs(free):
        if size >= k:
            return off
    return None


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_pool_matches_first_fit_model(driver, seed):
    rng = np.random.default_rng(seed)
    size = int(rng.integers(200, 2000))
    free = np.ones(size, bool)
    live, script, expect = [], [f"init {size}"], ["ok"]
    used = peak = 0
    checks = []
    for step in range(600):
        if live and (rng.random() < 0.45 or len(live) > 20):
            off, n = live.pop(int(rng.integers(len(live))))
            free[off:off + n] = True
            used -= n
            script.append(f"release {off} {n}")
            expect.append("ok")
        else:
            n = int(rng.integers(1, size // 4))
            off = _first_fit(free, n)
            script.append(f"alloc {n}")
            if off is None:
                expect.append("fail")
            else:
                expect.append(str(off))
                free[off:off + n] = False
                live.append((off, n))
                used += n
                peak = max(peak, used)
        if step % 7 == 0:
            runs = _runs(free)
            largest = max((s for _, s in runs), default=0)
            script.append("dump")
            expect.append(" ".join([str(used), str(peak), str(largest)] + [f"{o}:{s}" for o, s in runs]))
    out = subprocess.run([driver], input="\n".join(script) + "\n", capture_output=True, text=True, check=True)
    got = out.stdout.strip().split("\n")
    assert len(got) == len(expect)
    for k, (g, e) in enumerate(zip(got, expect)):
        assert g.strip() == e, f"command {k} ({script[k]}): {g!r} != {e!r}"


def test_pool_whole_and_empty(driver):
    script = "init 1024\nalloc 1024\nalloc 1\nrelease 0 1024\nalloc 1025\nalloc 512\nalloc 512\ndump\n" \
             "release 512 512\nrelease 0 512\ndump\ninit 0\nalloc 1\n"
    out = subprocess.run([driver], input=script, capture_output=True, text=True, check=True).stdout.split("\n")
    assert out[:8] == ["ok", "0", "fail", "ok", "fail", "0", "512", "1024 1024 0"]
    assert out[8:13] == ["ok", "ok", "0 1024 1024 0:1024", "ok", "fail"]
