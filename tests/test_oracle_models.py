"""Pins of the paper's memory-access and memory-footprint models against the
values the paper prints (tests/golden/paper_tables.json, each with its
table / equation)."""
import json
import os

import pytest

import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def reduction_pct(data, arch):
    pull = O.access_bytes(19, 8, 4, "pull", data, arch)
    aa = O.access_bytes(19, 8, 4, "aa", data, arch)
    return 100.0 * (1.0 - aa / pull)


@pytest.mark.parametrize("key,data,arch", [
    ("cpu_access_reduction_dense_pct", "dense", "cpu"),
    ("cpu_access_reduction_sparse_pct", "sparse", "cpu"),
    ("gpu_access_reduction_dense_pct", "dense", "gpu"),
])
def test_access_reductions_match_printed_tables(key, data, arch):
    assert round(reduction_pct(data, arch), 1) == GOLD[key]["value"]


def test_gpu_sparse_reduction_reading():
    # Table 2 prints 9.7 %; its own formula 1 - (2QB + (Q-1)/2 Bi)/(2QB + (Q-1)Bi)
    # gives 9.57 %.  We keep the formula (the byte count the roofline uses)
    # and accept the printed value as a rounding of it within 0.15 points.
    got = reduction_pct("sparse", "gpu")
    assert abs(got - 9.574) < 1e-3
    assert abs(got - GOLD["gpu_access_reduction_sparse_pct"]["value"]) < 0.15


def test_aa_memory_saving_matches_printed_value():
    pull = O.memory_bytes_per_cell(19, 8, 4, "sparse", 1.0)
    aa = O.memory_bytes_per_cell(19, 8, 4, "sparse_aa", 1.0)
    assert round(100.0 * (1.0 - aa / pull), 1) == GOLD["aa_memory_saving_sparse_pct"]["value"]


def test_memory_break_even_porosity():
    dense = O.memory_bytes_per_cell(19, 8, 4, "dense", 1.0)
    sparse_full = O.memory_bytes_per_cell(19, 8, 4, "sparse", 1.0)
    phi = dense / sparse_full
    g = GOLD["memory_break_even_porosity"]
    assert abs(phi - g["value"]) < g["tol"]


def test_aa_bytes_per_update_values():
    # the per-update byte counts the roofline uses (2QB + (Q-1)/2 Bi)
    assert O.access_bytes(19, 8, 4, "aa", "sparse", "gpu") == 340
    assert O.access_bytes(19, 8, 4, "pull", "sparse", "gpu") == 376
    assert O.access_bytes(19, 4, 4, "aa", "sparse", "gpu") == 188
    assert O.access_bytes(19, 2, 4, "aa", "sparse", "gpu") == 112
    assert O.access_bytes(27, 4, 4, "aa", "sparse", "gpu") == 268
