"""The oracle reproduces its committed trajectory on this host (regression pin)."""
import json
import os

import pytest

import golden_make


FIX = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "random_10k_oracle.json")


@pytest.mark.parametrize("i", range(3))
def test_oracle_trajectory_unchanged(i):
    want = json.load(open(FIX))["runs"][i]
    got = golden_make.trajectory(want["seed"])
    assert got == want


COARSE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "coarsen_10k_oracle.json")


@pytest.mark.parametrize("i", range(2))
def test_oracle_coarsening_unchanged(i):
    want = json.load(open(COARSE))["runs"][i]
    assert golden_make.coarsening(want["seed"]) == want
