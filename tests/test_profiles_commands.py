"""The ncu summaries under profiles/ each give the command that produced them. This checks that
every such command keeps the GPU clocks untouched (`--clock-control none`), runs bench.py with
options that bench.py still accepts, so that each summary can be reproduced from the tree, and
that every capture collecting more than kernel durations stays on a small case: one of bench.py's
profiling cases or a grid of at most 512^3, and at most three captured launches."""
import glob
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _commands(text):
    """ncu command lines of a summary, with backslash continuations joined."""
    joined = re.sub(r"\\\n\s*", " ", text)
    return [line.strip() for line in joined.splitlines() if line.strip().startswith("ncu ")]


def _bench_options():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True,
                         text=True, timeout=120, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    return set(re.findall(r"(--[a-z0-9][a-z0-9-]*)", out.stdout))


def test_profile_commands_are_reproducible():
    options = _bench_options()
    summaries = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert summaries
    for path in summaries:
        cmds = _commands(open(path).read())
        assert cmds, f"{os.path.basename(path)} gives no ncu command"
        for cmd in cmds:
            assert "--clock-control none" in cmd, (path, cmd)
            if "bench.py" in cmd:
                for opt in re.findall(r"(--[a-z0-9][a-z0-9-]*)", cmd.split("bench.py", 1)[1]):
                    assert opt in options, (os.path.basename(path), opt)


# bench.py --profile-case: each holds at most a few GB on the device (net512: the network at
# 512^3, about 2.4 GB)
SMALL_CASES = {"op384", "cg512", "var240", "robin200", "net512"}


def _collects_more_than_durations(cmd):
    if "--set" in cmd or "--section" in cmd:
        return True
    for group in re.findall(r"--metrics\s+(\S+)", cmd):
        if any(m != "gpu__time_duration.sum" for m in group.split(",")):
            return True
    return False


def test_profile_captures_stay_small():
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for cmd in _commands(open(path).read()):
            if not _collects_more_than_durations(cmd):
                continue
            name = os.path.basename(path)
            count = re.search(r"\s-c\s+(\d+)", cmd)
            assert count and int(count.group(1)) <= 3, (name, "capture at most three launches")
            tail = cmd.split("bench.py", 1)[1] if "bench.py" in cmd else ""
            case = re.search(r"--profile-case\s+(\S+)", tail)
            grid = re.search(r"--grid\s+(\d+)", tail)
            assert (case and case.group(1) in SMALL_CASES) or (grid and int(grid.group(1)) <= 512), \
                (name, "a capture beyond kernel durations must run a small case")
