"""Host logic of the served loop, compiled with g++ (no GPU involved): the
first-fit device-pool sub-allocator (csrc/pool.h), checked by
tests/c/pool_check.cpp against a byte map of the pool under seeded random
allocations and releases (first-fit offsets, no overlap, alignment, used
bytes, full merge on release); and the scheduler's policy rules
(csrc/serve_policy.h: eviction victim, half-pool batch bound, ready order,
the launch form of a batch), checked by tests/c/sched_check.cpp."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_first_fit_pool_against_a_byte_map(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "pool_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Wextra", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2003_12787_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "c", "pool_check.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")


# Plausible mistakes in the allocator; the byte-map check must catch each.
MUTANTS = {
    "no merge with the next free block":
        ("if (next != free_.end() && it->first + it->second == next->first) {", "if (false) {"),
    "no merge with the previous free block":
        ("if (prev->first + prev->second == it->first) {", "if (false) {"),
    "alloc without rounding up": ("n = pool_align_up(n);\n    for", "for"),
    "release does not return the bytes": ("used_ -= n;", ""),
    "block carved from the end of the free run":
        ("*off = it->first;\n        const size_t rest = it->second - n;\n"
         "        const size_t start = it->first + n;\n        free_.erase(it);\n"
         "        if (rest) free_[start] = rest;",
         "*off = it->first + it->second - n;\n        it->second -= n;\n"
         "        if (!it->second) free_.erase(it);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_allocator_mistakes_are_caught(tmp_path, name):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(os.path.join(ROOT, "paper_2003_12787_gb300", "csrc", "pool.h")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, name
    (tmp_path / "pool.h").write_text(src.replace(old, new, 1))
    exe = tmp_path / "pool_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", str(tmp_path),
                    os.path.join(ROOT, "tests", "c", "pool_check.cpp"), "-o", str(exe)],
                   check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "mismatch" in r.stdout, (name, r.stdout)


def _compile_and_run(tmp_path, source, include_dir, werror=True):
    exe = tmp_path / "check"
    flags = ["-Wall", "-Wextra"] + (["-Werror"] if werror else [])
    subprocess.run(["g++", "-std=c++17", "-O1", *flags, "-I", include_dir,
                    os.path.join(ROOT, "tests", "c", source), "-o", str(exe)], check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)


def test_scheduler_rules_against_their_literal_reading(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    r = _compile_and_run(tmp_path, "sched_check.cpp",
                         os.path.join(ROOT, "paper_2003_12787_gb300", "csrc"))
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout + r.stderr


SCHED_MUTANTS = {
    "busy simulations may be evicted": ("c.busy || ", ""),
    "no preference for simulations without requests":
        ("if (pass == 0 && !c.pending.empty()) continue;", ""),
    "most recently used instead of least": ("c.last_used < sims[victim].last_used",
                                            "c.last_used > sims[victim].last_used"),
    "no half-pool bound": ("return batch_bytes + bytes <= budget / 2;", "return true;"),
    "no age bound": ("return now - sims[i].pending.front().t_arrival >= age_bound;", "return false;"),
    "resident ones last": ("if (!aged(i) && sims[i].resident) out->push_back(i);\n  for (int i : ready)\n    if (!aged(i) && !sims[i].resident)",
                           "if (!aged(i) && !sims[i].resident) out->push_back(i);\n  for (int i : ready)\n    if (!aged(i) && sims[i].resident)"),
    "FIFO policy reordered": ("if (policy == 0) {", "if (policy == 2) {"),
    "N = 12 rule dropped": ("(work > threshold_ms || (N[k] == 12 && !curvilinear[k]))", "(work > threshold_ms)"),
    "threshold compared the wrong way": ("(work > threshold_ms ||", "(work < threshold_ms ||"),
    "curvilinear weight missing": ("(curvilinear ? 1.7 : 1.0)", "1.0"),
    "per-set instead of per-batch work": ("out[k] = (work > threshold_ms ||",
                                          "out[k] = (step_work_ms(N[k], E[k], curvilinear[k] != 0) > threshold_ms ||"),
}


@pytest.mark.parametrize("name", sorted(SCHED_MUTANTS))
def test_planted_scheduler_mistakes_are_caught(tmp_path, name):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(os.path.join(ROOT, "paper_2003_12787_gb300", "csrc", "serve_policy.h")).read()
    old, new = SCHED_MUTANTS[name]
    assert old in src, name
    (tmp_path / "serve_policy.h").write_text(src.replace(old, new, 1))
    r = _compile_and_run(tmp_path, "sched_check.cpp", str(tmp_path), werror=False)
    assert r.returncode != 0 and "mismatch" in r.stdout, (name, r.stdout + r.stderr)
