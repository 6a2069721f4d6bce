"""The ncu summaries under profiles/ give the command that made them, and it runs committed
files only: every `python ...` entry point they name exists in the repository."""
import glob
import os
import re

from conftest import ROOT


def test_profile_commands_name_committed_entry_points():
    files = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
    assert files
    for path in files:
        text = open(path).read()
        assert "--clock-control none" in text, path            # every ncu command keeps the clocks
        cmds = re.findall(r"python\s+(-m\s+[\w.]+|[\w./-]+\.py)", text)
        assert cmds, path
        for c in cmds:
            if c.startswith("-m"):
                mod = c.split()[1].replace(".", os.sep)
                ok = os.path.exists(os.path.join(ROOT, mod + ".py")) or os.path.isdir(os.path.join(ROOT, mod))
                assert ok, (path, c)
            else:
                assert os.path.exists(os.path.join(ROOT, c)), (path, c)
        assert "_work" not in text, path
