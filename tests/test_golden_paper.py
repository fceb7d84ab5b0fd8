"""The paper's printed constants (tests/golden/paper_constants.json) against the library and the byte model."""
import json
import os

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_library_defaults_follow_the_paper():
    import paper_1811_03852_gb300 as hz

    p = hz.default_params()
    assert p.restart == GOLD["restart_iterations"]["value"]
    # FP32 inner solves stop at the paper's latest operational tolerance (R_c >> eps_32, Sec. 3)
    assert p.inner_tol == 0.0  # 0 selects the mode default, 1e-4 for the mixed solver
    assert 1e-4 in GOLD["operational_tolerances"]["value"]


def test_working_set_arithmetic_fixes_the_element_sizes():
    # the byte model of the roofline uses 4 B per FP32 and 8 B per FP64 value, as the paper's working set does
    n = GOLD["working_set_values"]["value"]
    assert n == 111720 * 10
    assert n * 4 == GOLD["working_set_bytes_fp32"]["value"]
    assert n * 8 == GOLD["working_set_bytes_fp64"]["value"]


def test_table1_mixed_speedup_is_context():
    t3 = GOLD["table1_seconds_1e-3"]
    t4 = GOLD["table1_seconds_1e-4"]
    assert 1.6 < t3["double"] / t3["mixed"] < 1.8 and 1.6 < t4["double"] / t4["mixed"] < 1.8
