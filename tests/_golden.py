"""Reads the fixtures of tests/golden/: values printed in the paper, one file per table or
worked example, each file citing its source in '#' comment lines.  A data line is a key
followed by one or more numbers."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name: str) -> dict:
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            nums = [float(v) if any(c in v for c in ".e") else int(v) for v in vals]
            out[key] = nums[0] if len(nums) == 1 else nums
    return out
