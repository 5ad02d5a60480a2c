"""Numbers the paper prints (tests/golden/paper_values.json, each with its citation)."""
import json
import os

from oracle import dense

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_rho_for_table1_parameters():
    """Sec. 5: rho >= 1 and rho -> 1 as mu -> 0 for the kernel masses of Table 1."""
    r_bmw = dense.rho_from_mu(GOLD["table1_BMW_mu"]["value"], GOLD["table1_BMW_m0_ker"]["value"])
    r_jf = dense.rho_from_mu(GOLD["table1_JF_mu"]["value"], -1.0)
    assert 1.0 < r_bmw < 1.011 and 1.0 < r_jf < 1.016
    assert dense.rho_from_mu(1e-9, -1.0) - 1.0 < 1e-8


def test_fixture_is_cited():
    for k, v in GOLD.items():
        if not k.startswith("_"):
            assert v["cite"] and "value" in v
