"""The committed ncu summaries: short text, each with the command that made it.

Every ncu invocation in a summary leaves the GPU clocks alone
(``--clock-control none``), and the commands run only files of this
repository (``bench.py`` or a module of the package).
"""
import os
import re

import pytest

PROFILES = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "profiles")
NAMES = sorted(f for f in os.listdir(PROFILES) if not f.startswith("."))


def test_profiles_are_short_text_summaries():
    assert NAMES, "no committed summaries"
    for name in NAMES:
        assert name.endswith((".txt", ".md")), name
        assert os.path.getsize(os.path.join(PROFILES, name)) < 16 * 1024, name


@pytest.mark.parametrize("name", NAMES)
def test_each_summary_gives_its_command(name):
    txt = open(os.path.join(PROFILES, name)).read()
    assert re.search(r"^\s*commands?\b", txt, re.M), f"{name}: no command line"


@pytest.mark.parametrize("name", NAMES)
def test_ncu_invocations_keep_the_clocks(name):
    for line in open(os.path.join(PROFILES, name)):
        invocation = "ncu --" in line and any(k in line for k in ("--csv", " -o ", "-k regex", "--log-file", " -c "))
        if invocation:
            assert "--clock-control none" in line, f"{name}: {line.strip()}"


@pytest.mark.parametrize("name", NAMES)
def test_commands_run_repository_files_only(name):
    for line in open(os.path.join(PROFILES, name)):
        for m in re.finditer(r"\bpython3?\s+(-m\s+(\S+)|(\S+\.py))", line):
            module, script = m.group(2), m.group(3)
            if module:
                assert module.startswith("paper_1902_10559_gb300."), f"{name}: {line.strip()}"
            else:
                assert script == "bench.py", f"{name}: {line.strip()}"
