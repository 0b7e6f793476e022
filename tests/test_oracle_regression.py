"""The oracle against its stored regression fixture (tests/golden/): the
same small seeded cases, recomputed, to 1e-12 relative (the oracle is
independent of its thread count; the margin covers a compiler's choice of
fused multiply-adds)."""
import json
import os
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402

with open(os.path.join(HERE, "golden", "oracle_regression.json")) as fh:
    GOLDEN = json.load(fh)


@pytest.mark.parametrize("case", sorted(GOLDEN))
def test_oracle_matches_stored_fixture(case):
    got = make_golden.CASES[case]()
    want = GOLDEN[case]
    assert sorted(got) == sorted(want)
    for step, rec in want.items():
        for k, v in rec.items():
            g = got[step][k]
            scale = max(abs(v), 1e-300)
            # gauss residuals are round-off-sized: compare them absolutely
            tol = 1e-12 * (1.0 if k == "gauss" else scale)
            assert abs(g - v) <= max(tol, 1e-15 if k == "gauss" else 0.0), (case, step, k, g, v)
