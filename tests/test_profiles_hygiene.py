"""The committed profile summaries (no GPU): each is a short text file that
names the command it came from, every ncu command in it leaves the GPU
clocks alone (--clock-control none), and profiles/ holds no raw reports."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROF = os.path.join(ROOT, "profiles")


def test_profiles_are_short_text_summaries():
    names = sorted(os.listdir(PROF))
    assert names
    for n in names:
        assert n.endswith((".md", ".txt", ".json")), n
        assert os.path.getsize(os.path.join(PROF, n)) < 16 * 1024, n


def test_every_ncu_command_keeps_the_clocks_unlocked():
    for n in sorted(os.listdir(PROF)):
        if not n.endswith(".md"):
            continue
        text = open(os.path.join(PROF, n)).read()
        blocks = re.findall(r"```(.*?)```", text, flags=re.S)
        assert blocks, f"{n}: no command block"
        cmds = [c for b in blocks for c in re.split(r"&&|;\s*done", b.replace("\\\n", " ")) if "ncu " in c]
        assert cmds, f"{n}: no ncu command"
        for c in cmds:
            assert "--clock-control none" in c, f"{n}: {c.strip()[:80]}"
