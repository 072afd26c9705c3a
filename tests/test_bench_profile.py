"""The benchmark's tie between the committed ncu summary and the kernel source (CPU): the
frames kernel's source sections are found, the summary carries its hash, the DRAM traffic
of one launch and the launch size it was captured at, and a summary taken on another
source gives no traffic figure."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_profile_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_kernel_sections_found():
    b = _bench()
    sha = b.frames_kernel_sha()
    assert sha is not None and re.fullmatch(r"[0-9a-f]{64}", sha)


def test_summary_fields_parse():
    text = open(os.path.join(ROOT, "profiles", "frames_kernel_pilatus6m.txt")).read()
    assert re.search(r"source_sha256:\s*[0-9a-f]{64}", text)
    t = re.search(r"traffic_bytes_per_launch_full:\s*([0-9]+)", text)
    f = re.search(r"capture_frames_per_launch:\s*([0-9]+)", text)
    assert t and f and int(t.group(1)) > 0 and int(f.group(1)) > 0
    # the command that made it is written out
    assert "ncu --set full --clock-control none" in text


def test_other_source_gives_no_traffic(tmp_path, monkeypatch):
    b = _bench()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "frames_kernel_pilatus6m.txt").write_text(
        "source_sha256: " + "0" * 64 + "\ntraffic_bytes_per_launch_full: 123\ncapture_frames_per_launch: 64\n")
    monkeypatch.setattr(b, "ROOT", str(tmp_path))
    monkeypatch.setattr(b, "frames_kernel_sha", lambda: "1" * 64)
    assert b.ncu_traffic() is None
    monkeypatch.setattr(b, "frames_kernel_sha", lambda: "0" * 64)
    assert b.ncu_traffic() == (123.0, 64)


def test_profile_commands_run_committed_options():
    """Every bench.py command written in a profile summary parses with the benchmark's own
    options (the summaries name committed files and flags only)."""
    b = _bench()
    found = 0
    for name in sorted(os.listdir(os.path.join(ROOT, "profiles"))):
        text = open(os.path.join(ROOT, "profiles", name)).read().replace("\\\n", " ")
        for line in text.splitlines():
            if "python bench.py" not in line:
                continue
            args = line.split("python bench.py", 1)[1].split()
            b.parse(args)  # SystemExit on an unknown option
            found += 1
    assert found >= 4
