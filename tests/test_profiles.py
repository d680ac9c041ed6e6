"""The committed ncu summaries stay reproducible (CPU): every summary gives
its command in a code block; every bench.py invocation there parses with
today's bench arguments; every ncu command leaves the GPU clocks alone
(--clock-control none); profiles/ holds text only."""
from __future__ import annotations

import glob
import importlib.util
import os
import re
import shlex

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_parser():
    spec = importlib.util.spec_from_file_location("bench_for_tests", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build_parser()


def _commands(path):
    text = open(path).read()
    out = []
    for block in re.findall(r"```[a-z]*\n(.*?)```", text, re.S):
        out += [ln.strip() for ln in block.replace("\\\n", " ").splitlines() if ln.strip()]
    return out


def test_profiles_are_text_summaries():
    for path in glob.glob(os.path.join(ROOT, "profiles", "*")):
        assert os.path.splitext(path)[1] in (".md", ".txt", ".json"), path
        assert os.path.getsize(path) < 64 * 1024, path


def test_profile_commands_parse_and_keep_clocks():
    parser = _bench_parser()
    summaries = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert summaries
    for path in summaries:
        cmds = _commands(path)
        assert any("bench.py" in c for c in cmds), path
        for c in cmds:
            toks = shlex.split(c)
            if toks and toks[0] == "ncu":
                assert "--clock-control" in toks and toks[toks.index("--clock-control") + 1] == "none", \
                    (path, c)
            if "bench.py" in c:
                i = max(k for k, t in enumerate(toks) if t.endswith("bench.py"))
                parser.parse_args(toks[i + 1:])  # exits (SystemExit) on an unknown flag
