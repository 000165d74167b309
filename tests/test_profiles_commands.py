"""The ncu summaries under profiles/ each give the command that produced them. This checks that
every such command keeps the GPU clocks untouched (`--clock-control none`) and runs bench.py with
options that bench.py still accepts, so that each summary can be reproduced from the tree."""
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
