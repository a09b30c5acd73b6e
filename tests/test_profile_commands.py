"""Every capture summary under profiles/ names the command that made it, and
that command runs files of this repository only: the capture driver's modes
and the seeded workloads it names exist (checked on CPU, nothing is run)."""
import os
import re

from paper_2605_04735_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")
MODES = {"apply", "apply64", "applydw", "solve", "simp", "batch", "serving"}


def summaries():
    return sorted(os.path.join(PROFILES, f) for f in os.listdir(PROFILES) if f.endswith(".md"))


def test_every_summary_gives_its_command():
    for path in summaries():
        text = open(path).read()
        assert "```" in text and ("ncu " in text or "bench.py" in text), path
        assert "--clock-control none" in text, path  # no capture locks the clocks


def test_capture_commands_name_existing_modes_and_workloads():
    src = open(os.path.join(ROOT, "paper_2605_04735_gb300", "profile_run.py")).read()
    for mode in MODES:
        assert f'"{mode}"' in src, mode
    seen = 0
    for path in summaries():
        for mode, arg in re.findall(r"profile_run (\w+) (\w+)", open(path).read()):
            assert mode in MODES, (path, mode)
            if mode != "serving":
                assert arg in I.WORKLOADS, (path, arg)
            seen += 1
    assert seen > 0
