"""Every profile summary the design notes, the README and bench.py name is
committed, and every committed summary gives the command that made it (CPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_named_profiles_exist():
    names = set()
    for f in ("DESIGN.md", "README.md", "bench.py"):
        names |= set(re.findall(r"profiles/([A-Za-z0-9_]+\.(?:md|json))", open(os.path.join(ROOT, f)).read()))
    assert names
    missing = sorted(n for n in names if not os.path.exists(os.path.join(ROOT, "profiles", n)))
    assert not missing, missing


def test_profiles_give_their_commands():
    for n in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        if n.endswith(".md"):
            text = open(os.path.join(ROOT, "profiles", n)).read()
            assert "ncu " in text and "--clock-control none" in text, n
            assert "bench.py" in text, n
