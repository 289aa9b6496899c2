"""The committed profile summaries stay consistent with the sources they
describe (CPU only): every DRAM-traffic entry that bench.py may report as
roofline.traffic carries the hash of the current kernel sources, uses the key
format bench.py looks up, and lies between the algorithmic bytes and a small
multiple of them; every ncu command in the summaries leaves the GPU clocks
alone."""
import importlib.util
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


SWEEP_KEY = re.compile(r"^(f32|bf16):(k|u):(adv|noadv):v-?\d+:d\d+:\d+x\d+x\d+$")
CG_KEY = re.compile(r"^implicit:(k|u):cg_iteration$")


def test_traffic_entries_match_the_current_kernels():
    bench = _bench()
    with open(os.path.join(PROFILES, "traffic.json")) as f:
        entries = json.load(f)
    assert entries
    for key, e in entries.items():
        if SWEEP_KEY.match(key):
            assert e["kernel_hash"] == bench.kernel_hash(), key
            measured, algorithmic = e["bytes_per_launch"], e["algorithmic_bytes_per_launch"]
            # the cells of the key's shape at the key's bytes a cell
            storage, cond = key.split(":")[:2]
            nx, ny, nz = (int(v) for v in key.split(":")[-1].split("x"))
            assert algorithmic == bench.bytes_per_cell(storage == "bf16", cond == "k") * nx * ny * nz, key
            assert isinstance(e.get("zchunk", 0), int)
        elif CG_KEY.match(key):
            assert e["kernel_hash"] == bench.cg_kernel_hash(), key
            measured, algorithmic = e["bytes_per_iteration"], e["algorithmic_bytes_per_iteration"]
        else:
            raise AssertionError(f"unknown traffic key {key}")
        # DRAM bytes of a launch: a little below the algorithmic bytes is
        # possible (writes still in L2 when the launch ends), far above it
        # would be a stale or mislabelled capture
        assert 0.9 * algorithmic <= measured <= 1.5 * algorithmic, (key, measured / algorithmic)
        assert "ncu" in e["source"]


def test_every_ncu_command_leaves_the_clocks_alone():
    names = [n for n in os.listdir(PROFILES) if n.endswith((".md", ".txt"))]
    assert names
    for name in names:
        with open(os.path.join(PROFILES, name)) as f:
            text = f.read()
        # an ncu command may continue over several lines (trailing backslash)
        joined = re.sub(r"\\\n\s*", " ", text)
        for line in joined.splitlines():
            if re.search(r"(^|\s|\$\()ncu\s+(?!-i\b)", line) and "--" in line:
                assert "--clock-control none" in line or "$M" in line or "$SEC" in line, (name, line)
        if "$M" in joined or "$SEC" in joined:
            for var in ("M", "SEC"):
                m = re.search(rf'^{var}="([^"]*)"', joined, re.M)
                if m:
                    assert "--clock-control none" in m.group(1) or "--clock-control none" in joined, (name, var)


def test_profiles_hold_text_only():
    for name in os.listdir(PROFILES):
        assert name.endswith((".md", ".txt", ".json")), name
