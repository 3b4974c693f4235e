"""The committed profile summaries stay consistent with the sources: the DRAM
traffic that bench.py reports is read from a summary valid only for one
pair.cu, and every summary names the command that produced it."""
import hashlib
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_pair_traffic_summary_matches_pair_source():
    src = open(os.path.join(ROOT, "paper_2104_10231_gb300", "csrc", "pair.cu"), "rb").read()
    sha = hashlib.sha256(src).hexdigest()[:16]
    vals = {}
    for line in open(os.path.join(PROFILES, "pair_neopentane_1M.txt")):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    assert vals["pair_cu_sha256_16"] == sha, "pair.cu changed since its DRAM traffic was captured"
    assert 1e8 < float(vals["dram_bytes_plain_launch_full_size"]) < float(vals["dram_bytes_pruning_launch_full_size"])


def test_profile_summaries_give_their_commands():
    names = sorted(os.listdir(PROFILES))
    assert names, "no profile summaries"
    for name in names:
        path = os.path.join(PROFILES, name)
        assert name.endswith((".md", ".txt")), name
        assert os.path.getsize(path) < 16_000, name
        text = open(path).read()
        assert "ncu" in text and "--clock-control none" in text, name
        # the commands run committed files only
        for script in re.findall(r"python (\S+\.py)", text):
            assert os.path.exists(os.path.join(ROOT, script)), (name, script)
        assert "_work" not in text, name
