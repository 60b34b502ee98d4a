"""The ncu summaries under profiles/ that bench.py reads DRAM traffic from.

Each such summary records the hash of the kernel sources it was captured on.
bench.py reports its traffic only while the sources still hash to that value,
so a kernel edited without a new capture reports `traffic: null`.  These tests
fail first, on CPU, so that the capture is redone with the change.  They also
check that every summary states the command that made it, and that the command
runs committed files only."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

TRAFFIC_PROFILES = [
    (bench.PROFILE_SUMMARY, bench.PAIR_SOURCES),
    (bench.PROFILE_SUMMARIES["f16"], bench.PAIR_SOURCES),
    (bench.PROFILE_SUMMARIES["bf16"], bench.PAIR_SOURCES),
    (bench.BATCH_PROFILE, bench.BATCH_SOURCES),
    (bench.SWEEP_PROFILE, bench.SWEEP_SOURCES),
]


@pytest.mark.parametrize("summary,sources", TRAFFIC_PROFILES, ids=lambda v: os.path.basename(v) if isinstance(v, str) else None)
def test_traffic_summary_matches_the_kernel_sources(summary, sources):
    text = open(summary).read()
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    assert m, "no kernel_source_hash line in " + summary
    assert m.group(1) == bench.kernel_source_hash(sources), (
        "kernel sources changed since %s was captured: capture it again" % os.path.basename(summary))
    t = bench.profiled_traffic(summary, sources)
    assert t is not None and t > 0


def test_traffic_is_close_to_the_algorithmic_bytes():
    """Traffic well above the algorithmic bytes would mean re-reads; well below,
    a capture of some other kernel or size."""
    import numpy as np
    from paper_1808_04406_gb300 import inputs
    sides = np.asarray(inputs.batched_run_sizes(512)[0]).astype(np.int64)
    cases = [
        (bench.PROFILE_SUMMARY, bench.PAIR_SOURCES, 2 * 27 * 4 * 256 ** 3),
        (bench.PROFILE_SUMMARIES["f16"], bench.PAIR_SOURCES, 2 * 27 * 2 * 256 ** 3),
        (bench.PROFILE_SUMMARIES["bf16"], bench.PAIR_SOURCES, 2 * 27 * 2 * 256 ** 3),
        (bench.SWEEP_PROFILE, bench.SWEEP_SOURCES, 2 * 9 * 8 * 4096 ** 2),
        (bench.BATCH_PROFILE, bench.BATCH_SOURCES, 2 * 9 * 2 * int((sides ** 2).sum())),
    ]
    for summary, sources, algorithmic in cases:
        t = bench.profiled_traffic(summary, sources)
        assert 0.9 * algorithmic <= t <= 1.1 * algorithmic, (summary, t, algorithmic)


def test_every_summary_gives_its_commands_on_committed_files():
    names = sorted(f for f in os.listdir(os.path.join(ROOT, "profiles")) if f.endswith(".md"))
    assert names
    for name in names:
        text = open(os.path.join(ROOT, "profiles", name)).read()
        # indented command lines, with backslash continuations joined
        joined, cur = [], ""
        for ln in text.splitlines():
            if ln.startswith("    ") or cur:
                cur += " " + ln.strip().rstrip("\\")
                if not ln.rstrip().endswith("\\"):
                    joined.append(cur)
                    cur = ""
        cmds = [c for c in joined if re.search(r"\b(python|ncu)\b", c)]
        assert cmds, name + " gives no command"
        for ln in cmds:
            for script in re.findall(r"python\s+([\w./-]+\.py)", ln):
                assert os.path.exists(os.path.join(ROOT, script)), (name, script)
            assert "_work" not in ln, (name, ln)
            if "ncu " in ln:
                assert "--clock-control none" in ln, (name, ln)
