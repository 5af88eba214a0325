"""The planted-mistake checker (tests/oracle_mutations.py) stays usable: each of its entries
still names text that occurs exactly once in the oracle, and the harness reports a planted
mistake as caught (the full sweep runs by hand; it takes minutes)."""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

import oracle_mutations as M  # noqa: E402


def test_every_entry_matches_the_oracle_once():
    text = open(M.ORACLE).read()
    bad = [(name, text.count(old)) for name, _, old, _ in M.MUTATIONS if text.count(old) != 1]
    assert not bad, bad
    names = [m[0] for m in M.MUTATIONS]
    assert len(names) == len(set(names))


def test_harness_catches_a_planted_sign_error():
    text = open(M.ORACLE).read()
    name, _, old, new = next(m for m in M.MUTATIONS if m[0] == "L-sign")
    assert M.run_pins(text.replace(old, new)) is False
