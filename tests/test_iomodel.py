"""The byte/FLOP model reproduces every number the paper prints for it."""
from __future__ import annotations

import json
import os

import pytest

from paper_2606_26439_gb300 import iomodel as io

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_io_model.json")))


def test_ai_table_bytes_exact():
    g = GOLD["ai_example"]
    args = (g["B"], g["nq"], g["nd"], g["d"])
    assert io.io_naive(*args) == g["io_naive_bytes"]
    assert io.io_fused(*args) == g["io_fused_bytes"]
    fl = io.flops_paper(*args)
    assert round(fl / io.io_naive(*args), 1) == g["ai_naive"]
    assert round(fl / io.io_fused(*args), 1) == g["ai_fused"]
    assert round(io.io_naive(*args) / io.io_fused(*args), 1) == g["io_reduction"]


def test_ai_nq64_reduction():
    g = GOLD["ai_nq64"]
    args = (g["B"], g["nq"], g["nd"], g["d"])
    assert round(io.io_naive(*args) / io.io_fused(*args), 1) == g["io_reduction"]


def test_h100_crossover():
    g = GOLD["h100_crossover"]
    assert round(g["tflops"] / g["tbps"]) == g["flop_per_byte"]


def test_pq_io_table_exact():
    g = GOLD["pq_io_table"]
    dec = io.io_pq_decompress(g["B"], g["nq"], g["nd"], g["d"], g["M"])
    fus = io.io_pq_fused(g["B"], g["nq"], g["nd"], g["M"], g["K"])
    assert dec == g["decompress_bytes"]
    assert fus == g["fused_bytes"]
    assert round(dec / fus, 1) == g["reduction"]


@pytest.mark.parametrize("row", GOLD["profiling_table"]["rows"])
def test_profiling_table_uses_theorem1_bytes(row):
    """The profiling table's GB/s is Theorem 1's bytes (B*4 output) over the
    latency, and its TFLOP/s is the 2 B Nq Nd d dot-product FLOPs over it
    (to the rounding of the printed latency)."""
    g = GOLD["profiling_table"]
    B, nq, nd, d = row["B"], g["nq"], g["nd"], g["d"]
    t = row["ms"] * 1e-3
    gbs = io.io_theorem1(B, nq, nd, d) / t / 1e9
    # the printed latency has 2-3 significant digits: allow its rounding
    rel_t = 0.0005 / row["ms"]
    assert abs(gbs - row["gbs"]) <= row["gbs"] * rel_t + 1.0
    tf = io.flops_dot(B, nq, nd, d) / t / 1e12
    assert abs(tf - row["tflops"]) <= row["tflops"] * rel_t + 0.1
    # the printed percentage is of the unrounded GB/s: within 0.1 point
    assert abs(100 * row["gbs"] / g["peak_gbs"] - row["pct"]) <= 0.1


@pytest.mark.parametrize("row", GOLD["batch_scaling_table"]["rows"])
def test_batch_scaling_table(row):
    g = GOLD["batch_scaling_table"]
    t = row["ms"] * 1e-3
    gbs = io.io_theorem1(row["B"], g["nq"], g["nd"], g["d"]) / t / 1e9
    assert abs(gbs - row["gbs"]) <= row["gbs"] * 0.005 / row["ms"] + 1.0
    assert abs(row["B"] / t / 1e6 - row["mdocs"]) <= 0.1 + row["mdocs"] * 0.005 / row["ms"]


def test_headline_fraction():
    g = GOLD["headline"]
    assert round(100 * g["gbs"] / g["peak_gbs"], 1) == g["pct"]


def test_packed_alg_bytes_reduces_to_theorem1():
    """With fixed-length documents and no metadata, the packed algorithmic
    byte count equals Theorem 1 with BQ = Nq."""
    B, nq, nd, d = 10000, 32, 128, 128
    packed = io.dense_alg_bytes(B * nd, B, 1, nq, d, 2) - B * io.META_BYTES_PER_CAND
    assert packed == io.io_theorem1(B, nq, nd, d)
