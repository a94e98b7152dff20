"""The committed ncu summaries under profiles/: each gives the full ncu command that made it,
with --clock-control none (ncu must not lock the GPU's clocks), runs only committed files of this
repository, and every source file and bench workload it names exists. Text checks on CPU."""
import glob
import os
import re

import pytest

from paper_2601_21310_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))


def test_profiles_exist():
    assert len(PROFILES) >= 5


@pytest.mark.parametrize("path", PROFILES, ids=[os.path.basename(p) for p in PROFILES])
def test_profile_states_its_command(path):
    text = open(path).read()
    assert "ncu " in text
    # every ncu command of the summary leaves the clocks alone
    cmds = re.findall(r"^[ \t`]*ncu --(?:[^\n]*\\\n)*[^\n]*", text, re.M)
    assert cmds, "no ncu command line"
    for cmd in cmds:
        assert "--clock-control none" in cmd, cmd[:80]
    # the programs it runs are committed files of this repository
    for script in set(re.findall(r"python ([\w./-]+\.py)", text)):
        assert os.path.exists(os.path.join(ROOT, script)), script
        assert not script.startswith("_work"), script
    for wl in set(re.findall(r"--workload ([\w]+)", text)):
        assert wl in synth.WORKLOADS or wl == "batched", wl
    # a committed traffic or issue figure names the source it was captured from
    for src in re.findall(r"^- source_file: (\S+)", text, re.M):
        assert os.path.exists(os.path.join(ROOT, src)), src
