"""The committed ncu summaries stay tied to the sources they describe.

* the gather/apply traffic summary names the sha256 prefix of the current
  train.cu, so the benchmark line's `roofline.traffic` is reported (it is
  null whenever the kernel source has changed since the counters were
  taken);
* every ncu command in a summary leaves the GPU clocks alone
  (`--clock-control none`) and runs committed files.
"""
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = os.path.join(ROOT, "profiles")


def test_traffic_summary_matches_the_kernel_source():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.measured_traffic() is not None


def test_ncu_commands_leave_the_clocks_alone():
    names = sorted(f for f in os.listdir(PROFILES) if f.endswith(".md"))
    assert names
    for name in names:
        text = open(os.path.join(PROFILES, name)).read()
        # join continued lines, then check each ncu invocation
        flat = re.sub(r"\\\n\s*", " ", text)
        for line in flat.splitlines():
            if re.search(r"(^|\s)ncu\s+--", line):
                assert "--clock-control none" in line, (name, line)
                assert "_work" not in line, (name, line)
