"""The bench line's capture-derived roofline fields (CPU).

`bench.py` reports `roofline.traffic` and `roofline.smem_pipe` from committed ncu
summaries under profiles/, each tied to the SHA-1 prefix of the kernel's source file at
capture time.  These checks keep those tables honest: every entry names a committed
profile that quotes the same source prefix and the same counter value, and a changed
source makes the bench report no number instead of a stale one.
"""
import os
import re

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _entries():
    for table in (bench.TRAFFIC, bench.SMEM_WAVEFRONTS):
        for key, (value, src, sha, profile) in table.items():
            yield table, key, value, src, sha, profile


def test_every_capture_entry_names_a_committed_profile_with_its_source_prefix():
    seen = 0
    for _, key, value, src, sha, profile in _entries():
        path = os.path.join(ROOT, profile)
        assert os.path.isfile(path), (key, profile)
        text = open(path, encoding="utf-8").read()
        assert f"`csrc/{src}`" in text, (key, profile)
        assert sha in text, (key, profile, sha)
        assert re.fullmatch(r"[0-9a-f]{12}", sha), sha
        assert value > 0
        seen += 1
    assert seen >= 3


def test_traffic_entries_match_the_profiles_read_plus_write():
    # the profiles state dram__bytes_read.sum and dram__bytes_write.sum in MB
    for key, (value, src, sha, profile) in bench.TRAFFIC.items():
        text = open(os.path.join(ROOT, profile), encoding="utf-8").read()
        mbs = [float(m) for m in re.findall(r"(\d+\.\d+) MB", text)]
        assert any(abs(a + b - value / 1e6) < 0.05 for a in mbs for b in mbs), (key, value)


def test_a_changed_source_reports_no_capture_number(monkeypatch):
    monkeypatch.setattr(bench, "source_sha1", lambda name: "000000000000")
    for kernel, workload in bench.TRAFFIC:
        nbytes, why = bench.traffic_of(kernel, workload)
        assert nbytes is None and "changed since" in why
    for kernel, workload in bench.SMEM_WAVEFRONTS:
        smem = bench.smem_pipe_of(kernel, workload, 0.05, 2070.0, 152)
        assert smem["wavefronts"] is None and "changed since" in smem["source"]


def test_smem_pipe_is_wavefronts_per_sm_clock():
    (kernel, workload), (wf, _, _, _) = next(iter(bench.SMEM_WAVEFRONTS.items()))
    ms, mhz, nsm = 0.05, 2000.0, 100
    smem = bench.smem_pipe_of(kernel, workload, ms, mhz, nsm)
    if smem["wavefronts"] is None:  # the source changed since the capture
        return
    assert abs(smem["frac"] - wf / (ms * 1e-3 * nsm * mhz * 1e6)) < 1e-12
    assert smem["peak"] == 1.0
