"""The profile summaries stay reproducible: each gives the command that made it, the
command runs committed files with arguments their current parsers accept, the ncu
capture re-runs exactly the plain command that exited 0 before it, and every ncu call
leaves the clocks alone (--clock-control none).  The README's example commands parse
the same way."""
import glob
import importlib.util
import os
import shlex
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def _commands(path):
    out = []
    for line in open(path):
        line = line.strip().strip("`")
        if line.startswith("python ") and "&& ncu " in line:
            out.append(line)
    return out


def _bench_parse(argv, monkeypatch):
    spec = importlib.util.spec_from_file_location("bench_for_profiles", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    spec.loader.exec_module(mod)
    monkeypatch.setattr(sys, "argv", ["bench.py"] + argv)
    return mod.parse()


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_command_is_reproducible(path, monkeypatch):
    import datagen
    from paper_2602_04551_b300 import profile_case

    cmds = _commands(path)
    assert cmds, "no command recorded"
    for cmd in cmds:
        plain, rest = cmd.split(" > ", 1)
        ncu = rest[rest.index("&& ncu ") + 3:]
        assert "--clock-control none" in ncu
        target = ncu[ncu.index(" python ") + 1:]
        assert target.strip() == plain.strip(), "the capture must re-run the plain command"
        tok = shlex.split(plain)
        if tok[:3] == ["python", "-m", "paper_2602_04551_b300.profile_case"]:
            a = profile_case.parser().parse_args(tok[3:])
        else:
            assert tok[:2] == ["python", "bench.py"], tok[:3]
            assert os.path.exists(os.path.join(ROOT, tok[1]))
            a = _bench_parse(tok[2:], monkeypatch)
        assert a.workload in datagen.CONFIGS


def test_readme_commands_parse(monkeypatch):
    """The commands the README shows run committed entry points with accepted arguments."""
    lines = []
    cont = ""
    for raw in open(os.path.join(ROOT, "README.md")):
        line = raw.split("#")[0].rstrip()
        if cont:
            line = cont + " " + line.strip()
            cont = ""
        if line.endswith("\\"):
            cont = line[:-1].strip()
            continue
        if line.strip().startswith("python "):
            lines.append(line.strip())
    assert any("bench.py" in l for l in lines)
    for cmd in lines:
        tok = shlex.split(cmd)
        if tok[:2] == ["python", "bench.py"]:
            _bench_parse(tok[2:], monkeypatch)
        elif tok[:3] == ["python", "-m", "pytest"]:
            assert os.path.isdir(os.path.join(ROOT, tok[3]))
        else:
            assert tok[:2] == ["python", "-m"], tok
            mod = tok[2].replace(".", os.sep)
            assert os.path.exists(os.path.join(ROOT, mod + ".py")), tok[2]
