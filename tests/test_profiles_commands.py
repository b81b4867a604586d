"""The commands quoted in profiles/ run committed files only: each bench.py
command parses with bench.py's own options, and each `python -m` command
names a module of this repository that defines every option it is given.
Runs on CPU (nothing is executed)."""
import glob
import os
import re
import shlex
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CMD = re.compile(r"python3? (?:-m [\w.]+|[\w/]+\.py)[^`|]*")


def quoted_commands():
    out = []
    for p in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(p).read().replace("\\\n", " ")
        for line in text.splitlines():
            for m in CMD.finditer(line):
                cmd = re.split(r"\s(?:>|&&|;)", m.group(0))[0].strip().rstrip(")")
                out.append((os.path.basename(p), cmd))
    return out


def test_profiles_quote_commands():
    assert len(quoted_commands()) >= 15


def test_bench_commands_parse(monkeypatch):
    import bench
    n = 0
    for name, cmd in quoted_commands():
        argv = shlex.split(cmd)
        if argv[1] != "bench.py":
            continue
        monkeypatch.setattr(sys, "argv", argv[1:])
        bench.parse()          # argparse exits on an unknown option or workload
        n += 1
    assert n >= 10


def test_module_commands_name_repository_modules_and_their_options():
    for name, cmd in quoted_commands():
        argv = shlex.split(cmd)
        if argv[1] != "-m":
            continue
        path = os.path.join(ROOT, *argv[2].split(".")) + ".py"
        assert os.path.exists(path), (name, cmd)
        src = open(path).read()
        for a in argv[3:]:
            if a.startswith("--"):
                opt = a.split("=")[0]
                assert f'"{opt}"' in src, (name, opt)
