"""Host logic of the batched plan, compiled with g++ (no GPU involved): how
sets are grouped into per-shape persistent launches, numbered and ordered,
and spread over graph branches (csrc/launch_groups.h), checked by
tests/c/launch_groups_check.cpp on seeded random inputs; planted mistakes in
the header must each fail that check."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2003_12787_gb300", "csrc", "launch_groups.h")
CHECK = os.path.join(ROOT, "tests", "c", "launch_groups_check.cpp")


def _build_and_run(tmp_path, include_dir, strict=True):
    exe = tmp_path / "launch_groups_check"
    flags = ["-Wall", "-Wextra", "-Werror"] if strict else []
    subprocess.run(["g++", "-std=c++17", "-O1", *flags, "-I", include_dir, CHECK, "-o", str(exe)],
                   check=True)
    return subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)


def test_launch_grouping_properties(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    r = _build_and_run(tmp_path, os.path.dirname(HEADER))
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok ")


# Plausible mistakes in the grouping; the check must catch each.
MUTANTS = {
    "offset taken after adding the set's units":
        ("      l.first_unit.push_back(l.count);\n      l.count += in[j].units;",
         "      l.count += in[j].units;\n      l.first_unit.push_back(l.count);"),
    "chunks one set too large": ("(int)built[g].sets.size() == max_sets", "(int)built[g].sets.size() == max_sets + 1"),
    "shortest launch first": ("return a.cost > b.cost;", "return a.cost < b.cost;"),
    "sets without units kept": ("if (done[j] || in[j].units <= 0 || in[j].key != in[i].key) continue;",
                                "if (done[j] || in[j].key != in[i].key) continue;"),
    "sets of another key mixed in": ("if (done[j] || in[j].units <= 0 || in[j].key != in[i].key) continue;",
                                     "if (done[j] || in[j].units <= 0) continue;"),
    "cost without the unit count": ("l.cost += in[j].unit_cost * (double)in[j].units;",
                                    "l.cost += in[j].unit_cost;"),
    "most loaded branch": ("std::min_element(load.begin(), load.end())", "std::max_element(load.begin(), load.end())"),
    "unstable order of ties": ("std::stable_sort(built.begin()", "std::sort(built.begin()"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_grouping_mistakes_are_caught(tmp_path, name):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    src = open(HEADER).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    (tmp_path / "launch_groups.h").write_text(src.replace(old, new))
    r = _build_and_run(tmp_path, str(tmp_path), strict=False)
    assert r.returncode != 0, f"mistake not caught: {name}"
