"""The stored full-size oracle results (tests/golden/fullsize_oracle.json,
written by make_golden.py --fullsize from the oracle alone) stay tied to
their inputs: the generators still produce the same pairs, and the stored
figures satisfy the identities that hold for any graph."""
from __future__ import annotations

import hashlib
import json
import os

import pytest

from paper_1907_09575_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fullsize_oracle.json")


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as f:
        return json.load(f)


def test_stored_results_satisfy_identities(gold):
    for name, g in gold.items():
        assert g["per_vertex_sum"] == 3 * g["total"], name       # each triangle has 3 vertices
        assert g["m"] <= g["num_pairs"], name
        assert g["max_outdeg"] <= g["max_deg"] < g["n"], name
        assert g["total"] <= g["wedges_jik"], name                # every triangle is one probe hit


def test_rmat_scale26_pairs_are_the_stored_ones(gold):
    g = gold["rmat-s26"]
    spec = inputs.rmat_graph(1, 26, 16)
    assert (spec.n, spec.num_pairs) == (g["n"], g["num_pairs"])
    src, dst = spec.generate()
    h = hashlib.sha256()
    h.update(src.astype("<i4", copy=False).tobytes())
    h.update(dst.astype("<i4", copy=False).tobytes())
    assert h.hexdigest() == g["pairs_sha256"]
