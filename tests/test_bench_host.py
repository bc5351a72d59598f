"""Host logic of bench.py that decides which ncu figures a run may use (no GPU).

The DRAM traffic of the contact pass comes from a committed ncu summary only
while the summary's hash equals this build's hash of the kernel's translation
unit: contact.cu, the repository headers it includes, and the nvcc flags.
"""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _copy_tree(tmp):
    for sub in ("paper_1906_05260_gb300/csrc", "include", "profiles"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(tmp, sub))


def test_unit_hash_follows_includes_only(tmp_path, monkeypatch):
    tmp = str(tmp_path)
    _copy_tree(tmp)
    monkeypatch.setattr(bench, "ROOT", tmp)
    h0 = bench.kernel_source_hash("contact.cu")
    assert h0 == bench.kernel_source_hash("contact.cu")
    csrc = os.path.join(tmp, "paper_1906_05260_gb300", "csrc")
    # a file outside the unit (not included by contact.cu) leaves the hash alone
    with open(os.path.join(csrc, "batch.cu"), "a") as f:
        f.write("\n// edit\n")
    assert bench.kernel_source_hash("contact.cu") == h0
    # a header two includes deep (contact.cu -> phases.cuh -> viper_device.cuh) changes it
    with open(os.path.join(csrc, "viper_device.cuh"), "a") as f:
        f.write("\n// edit\n")
    h1 = bench.kernel_source_hash("contact.cu")
    assert h1 != h0
    # and so does the public header, reached through viper_impl.h
    with open(os.path.join(tmp, "include", "viper.h"), "a") as f:
        f.write("\n/* edit */\n")
    assert bench.kernel_source_hash("contact.cu") != h1


def test_profile_traffic_used_only_for_the_captured_unit(tmp_path, monkeypatch):
    tmp = str(tmp_path)
    _copy_tree(tmp)
    monkeypatch.setattr(bench, "ROOT", tmp)
    prof = os.path.join(tmp, "profiles", "t.md")
    h = bench.kernel_source_hash("contact.cu")
    with open(prof, "w") as f:
        f.write(f"csrc sha256: {h}\n\ntraffic per candidate pair: 17.5 bytes per candidate pair\n")
    assert bench.profile_traffic("t.md", "per candidate pair") == 17.5
    assert bench.profile_traffic("t.md", "per pill") is None
    with open(os.path.join(tmp, "paper_1906_05260_gb300", "csrc", "contact.cu"), "a") as f:
        f.write("\n// edit\n")
    assert bench.profile_traffic("t.md", "per candidate pair") is None
    assert bench.profile_traffic("missing.md", "per candidate pair") is None


def test_committed_contact_summary_matches_this_build():
    """The committed summary was captured from the sources in the tree (else the
    bench would report no traffic and the summary's figures would be stale)."""
    assert bench.profile_traffic("contact_kernel_hair.md", "per candidate pair") is not None
