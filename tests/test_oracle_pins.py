"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

None of these checks re-derives a score with the oracle's own formula: they
use exact rational arithmetic on integer inputs, closed forms of special
cases, library routines for the cases that reduce to them (numpy matmul,
Python's sort), and invariants of the MaxSim definition (Eq. 1).  Each test
names the mistake it is there to catch.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _pack(docs):
    lengths = np.array([len(x) for x in docs], np.int32)
    offsets = synth.offsets_of(lengths)
    d = docs[0].shape[1] if len(docs[0]) else docs[1].shape[1]
    rows = [np.asarray(x, np.float64).reshape(-1, d) for x in docs]
    return np.concatenate(rows, 0), offsets, lengths


def _exact_maxsim(Q, X):
    """Eq. 1 with Python integers (inputs are integer-valued)."""
    best = []
    for qi in Q:
        vals = [sum(int(a) * int(b) for a, b in zip(qi, xj)) for xj in X]
        best.append(max(vals))
    return sum(best)


# ----------------------------------------------------------- element decode

def test_f16_decode_exhaustive():
    """All 65536 binary16 patterns decode as numpy's float16 (catches a wrong
    exponent bias, subnormal scale or sign handling)."""
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    want = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.f16_to_f64(int(b)) for b in bits])
    same = (got == want) | (np.isnan(got) & np.isnan(want))
    assert same.all()
    assert math.copysign(1.0, oracle.f16_to_f64(0x8000)) == -1.0


def test_bf16_decode_exhaustive():
    """All 65536 bfloat16 patterns decode as torch's bfloat16 -> float64."""
    torch = pytest.importorskip("torch")
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    want = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).double().numpy()
    got = np.array([oracle.bf16_to_f64(int(b)) for b in bits])
    same = (got == want) | (np.isnan(got) & np.isnan(want))
    assert same.all()


# ------------------------------------------------------------- dense MaxSim

@pytest.mark.parametrize("seed", range(6))
def test_dense_exact_integer_bruteforce(seed):
    """Small integer inputs: the fp64 oracle is exact, so it must equal the
    score computed with Python integers (catches a dropped term, a wrong
    index, sum/max swapped, or a transposed operand)."""
    g = np.random.default_rng(seed)
    nq, d = int(g.integers(1, 6)), int(g.integers(1, 9))
    docs = [g.integers(-7, 8, size=(int(g.integers(1, 6)), d)) for _ in range(5)]
    Q = g.integers(-7, 8, size=(nq, d))
    tok, off, ln = _pack(docs)
    cand = np.array([3, 0, 4, 1, 2, 2], np.int32)
    got = oracle.dense_scores(Q.astype(np.float64), tok, off, ln, cand)
    want = [_exact_maxsim(Q, docs[c]) for c in cand]
    assert got.tolist() == [float(w) for w in want]


def test_dense_fp16_integer_values_exact():
    """The same exactness through the fp16 decode path."""
    g = np.random.default_rng(11)
    Q = g.integers(-8, 9, size=(4, 16))
    docs = [g.integers(-8, 9, size=(n, 16)) for n in (1, 5, 9)]
    tok, off, ln = _pack(docs)
    cand = np.arange(3, dtype=np.int32)
    got = oracle.dense_scores(Q.astype(np.float16), tok.astype(np.float16), off, ln, cand)
    assert got.tolist() == [float(_exact_maxsim(Q, x)) for x in docs]


def test_dense_rational_random_floats():
    """Random fp64 inputs: within 1e-13 relative of the exact rational score."""
    g = np.random.default_rng(5)
    Q = g.standard_normal((3, 7))
    docs = [g.standard_normal((n, 7)) for n in (1, 4, 6)]
    tok, off, ln = _pack(docs)
    got = oracle.dense_scores(Q, tok, off, ln, np.arange(3, dtype=np.int32))
    for c, x in enumerate(docs):
        exact = sum(max(sum(Fraction(a) * Fraction(b) for a, b in zip(qi, xj)) for xj in x)
                    for qi in Q)
        assert abs(got[c] - float(exact)) <= 1e-13 * abs(float(exact)) + 1e-15


def test_dense_single_token_closed_form():
    """Nd = 1: sum_i q_i . x = (sum_i q_i) . x."""
    g = np.random.default_rng(2)
    Q = g.standard_normal((32, 128))
    x = g.standard_normal((1, 128))
    got = oracle.dense_scores(Q, x, np.array([0]), np.array([1], np.int32), np.array([0], np.int32))
    assert got[0] == pytest.approx(float(Q.sum(0) @ x[0]), rel=1e-12)


def test_dense_single_query_token_is_matvec_max():
    """Nq = 1: the score is the max entry of the matrix-vector product D q."""
    g = np.random.default_rng(3)
    q = g.standard_normal((1, 64))
    X = g.standard_normal((50, 64))
    got = oracle.dense_scores(q, X, np.array([0]), np.array([50], np.int32), np.array([0], np.int32))
    assert got[0] == pytest.approx(float((X @ q[0]).max()), rel=1e-12)


def test_dense_identity_document_is_rowmax():
    """Document = the d standard basis vectors: max_j q_i . e_j = max_t q_i[t],
    so the score is sum_i max_t q_i[t] (catches a transposed operand)."""
    g = np.random.default_rng(4)
    Q = g.standard_normal((9, 24))
    got = oracle.dense_scores(Q, np.eye(24), np.array([0]), np.array([24], np.int32),
                              np.array([0], np.int32))
    assert got[0] == pytest.approx(float(Q.max(1).sum()), rel=1e-13)


@pytest.mark.parametrize("dtype", ["f64", "f16"])
def test_dense_self_score_is_nq(dtype):
    """score(q, q) = Nq for unit-normalised q: by Cauchy-Schwarz each q_i's
    best match is itself, so the score is sum_i ||q_i||^2 -- exactly Nq up to
    fp64 rounding, and up to the stored norms' rounding for fp16."""
    q = synth.unit_rows(32, 128, 0)
    if dtype == "f16":
        q = q.astype(np.float16)
    qd = q.astype(np.float64)
    got = oracle.dense_scores(q, q, np.array([0]), np.array([32], np.int32), np.array([0], np.int32))
    assert got[0] == pytest.approx(float((qd * qd).sum()), rel=1e-13)
    assert abs(got[0] - 32.0) <= (1e-12 if dtype == "f64" else 32 * 2e-3)


def test_dense_permutation_invariant_bitwise():
    """Shuffling a document's tokens leaves the score bit-identical."""
    g = np.random.default_rng(6)
    Q = synth.unit_rows(32, 128, 6)
    X = synth.unit_rows(100, 128, 7)
    P = X[g.permutation(100)]
    tok = np.concatenate([X, P])
    got = oracle.dense_scores(Q, tok, np.array([0, 100]), np.array([100, 100], np.int32),
                              np.array([0, 1], np.int32))
    assert got[0] == got[1]


def test_dense_monotone_under_appended_tokens():
    """Appending tokens never lowers the score; appending a copy of an
    existing token leaves it unchanged."""
    Q = synth.unit_rows(16, 64, 8)
    X = synth.unit_rows(40, 64, 9)
    prefix = [oracle.dense_scores(Q, X, np.array([0]), np.array([n], np.int32),
                                  np.array([0], np.int32))[0] for n in range(1, 41)]
    assert all(b >= a for a, b in zip(prefix, prefix[1:]))
    Xd = np.concatenate([X, X[5:6]])
    dup = oracle.dense_scores(Q, Xd, np.array([0]), np.array([41], np.int32), np.array([0], np.int32))
    assert dup[0] == prefix[-1]


def test_dense_positive_scaling():
    """score(Q, 2^s D) = 2^s score(Q, D) exactly (max and sum commute with a
    positive power-of-two scale)."""
    Q = synth.unit_rows(8, 32, 10)
    X = synth.unit_rows(20, 32, 11)
    a = oracle.dense_scores(Q, X, np.array([0]), np.array([20], np.int32), np.array([0], np.int32))
    b = oracle.dense_scores(Q, 8.0 * X, np.array([0]), np.array([20], np.int32), np.array([0], np.int32))
    assert b[0] == 8.0 * a[0]


def test_dense_max_is_over_documents_tokens_not_queries():
    """A single strongly aligned token raises only the matching query
    token's max (catches max/sum taken over the wrong axis)."""
    Q = np.zeros((3, 4))
    Q[0, 0] = 1.0
    Q[1, 1] = 1.0
    Q[2, 2] = 1.0
    X = np.array([[5.0, 0, 0, 0], [0, 0, 0, 1.0], [0, 2.0, 0, 0]])
    got = oracle.dense_scores(Q, X, np.array([0]), np.array([3], np.int32), np.array([0], np.int32))
    # max_j: q0 -> 5, q1 -> 2, q2 -> 0
    assert got[0] == 7.0


def test_dense_packing_offsets_and_edge_cases():
    """Packed rows are addressed through offsets; empty documents score -inf;
    bad ids or row ranges score NaN; duplicate ids score identically."""
    Q = np.ones((2, 3))
    tok = np.arange(18, dtype=np.float64).reshape(6, 3)
    offsets = np.array([0, 2, 2, 5, 4], np.int64)
    lengths = np.array([2, 0, 3, 1, 3], np.int32)
    cand = np.array([0, 1, 2, 3, 5, -1, 4, 2], np.int32)
    got = oracle.dense_scores(Q, tok, offsets, lengths, cand)
    row_sums = tok.sum(1)
    assert got[0] == 2 * row_sums[0:2].max()
    assert got[1] == -math.inf
    assert got[2] == 2 * row_sums[2:5].max()
    assert got[3] == 2 * row_sums[5]
    assert math.isnan(got[4]) and math.isnan(got[5])
    assert math.isnan(got[6])  # rows 4..6 run past n_tokens = 6
    assert got[7] == got[2]
    neg = oracle.dense_scores(Q, tok, np.array([0]), np.array([-1], np.int32), np.array([0], np.int32))
    assert math.isnan(neg[0])


def test_dense_thread_count_does_not_change_results():
    """Candidates are independent; the result is bitwise the same for 1 or
    many OpenMP threads."""
    lengths = synth.lengths_uniform(300, 1, 40, 3)
    tok = synth.unit_rows(int(lengths.sum()), 48, 3, 1)
    off = synth.offsets_of(lengths)
    Q = synth.unit_rows(12, 48, 3, 2)
    cand = synth.candidates(300, 200, 3)
    n = oracle.max_threads()
    oracle.set_threads(1)
    a = oracle.dense_scores(Q, tok, off, lengths, cand)
    oracle.set_threads(max(n, 2))
    b = oracle.dense_scores(Q, tok, off, lengths, cand)
    oracle.set_threads(n)
    assert np.array_equal(a, b)


# -------------------------------------------------------------------- PQ

def test_pq_lut_exact_integer():
    """T[i][m][k] = q_i[m*dsub:(m+1)*dsub] . C[m][k] on integer inputs, with
    Python integers (catches a wrong sub-vector slice or codebook index)."""
    g = np.random.default_rng(20)
    nq, M, K, dsub = 3, 4, 5, 3
    Q = g.integers(-9, 10, size=(nq, M * dsub))
    C = g.integers(-9, 10, size=(M, K, dsub))
    lut = oracle.pq_lut(Q.astype(np.float64), C.astype(np.float32))
    for i in range(nq):
        for m in range(M):
            for k in range(K):
                want = sum(int(Q[i, m * dsub + t]) * int(C[m, k, t]) for t in range(dsub))
                assert lut[i, m, k] == want


def test_pq_lut_sum_equals_decompress_then_dot():
    """sum_m T[i][m][c_m] = q_i . d^_j (the ADC identity of Section 4.2), so
    the LUT path and the decompress path agree to fp64 rounding."""
    lengths = synth.lengths_uniform(60, 1, 30, 21)
    cb, codes, _, off, ln = synth.pq_corpus(lengths, M=16, K=256, dsub=8, seed=21)
    Q = synth.unit_rows(32, 128, 21, 3)
    cand = synth.candidates(60, 40, 21)
    a = oracle.pq_decompress_scores(Q, cb, codes, off, ln, cand)
    b = oracle.pq_lut_scores(oracle.pq_lut(Q, cb), codes, off, ln, cand)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_pq_exact_codebook_reproduces_dense():
    """When every token is exactly a concatenation of centroids (noise 0), PQ
    decompress-then-dot equals dense MaxSim on those tokens bit-for-bit."""
    lengths = synth.lengths_uniform(30, 1, 20, 22)
    cb, codes, x, off, ln = synth.pq_corpus(lengths, M=8, K=16, dsub=4, seed=22, noise=0.0)
    Q = synth.unit_rows(5, 32, 22, 3)
    cand = np.arange(30, dtype=np.int32)
    pq = oracle.pq_decompress_scores(Q, cb, codes, off, ln, cand)
    dense = oracle.dense_scores(Q, x.astype(np.float32), off, ln, cand)
    assert np.array_equal(pq, dense)


def test_pq_single_centroid_closed_form():
    """K = 1, all codes 0: every token is c = concat_m C[m][0], so the score
    is sum_i q_i . c = (sum_i q_i) . c whatever the length (>0)."""
    g = np.random.default_rng(23)
    M, dsub = 4, 8
    cb = g.standard_normal((M, 1, dsub)).astype(np.float32)
    codes = np.zeros((10, M), np.uint8)
    Q = g.standard_normal((6, M * dsub))
    c = cb[:, 0, :].reshape(-1).astype(np.float64)
    got = oracle.pq_decompress_scores(Q, cb, codes, np.array([0, 3]), np.array([3, 7], np.int32),
                                      np.array([0, 1], np.int32))
    want = float(Q.sum(0) @ c)
    np.testing.assert_allclose(got, [want, want], rtol=1e-12)
    lut_got = oracle.pq_lut_scores(oracle.pq_lut(Q, cb), codes, np.array([0, 3]),
                                   np.array([3, 7], np.int32), np.array([0, 1], np.int32))
    np.testing.assert_allclose(lut_got, [want, want], rtol=1e-12)


def test_pq_lut_scores_integer_table_exact():
    """An integer-valued fp32 table: every table sum is exact, so the score
    must equal the Python-integer evaluation of sum_i max_j sum_m T[i][m][c]
    (this is the exact reference used to check code gathering bit-for-bit)."""
    g = np.random.default_rng(24)
    nq, M, K = 8, 16, 256
    T = g.integers(-1000, 1001, size=(nq, M, K)).astype(np.float32)
    lengths = np.array([1, 4, 7, 33], np.int32)
    off = synth.offsets_of(lengths)
    codes = g.integers(0, K, size=(int(lengths.sum()), M)).astype(np.uint8)
    got = oracle.pq_lut_scores(T, codes, off, lengths, np.array([3, 2, 1, 0], np.int32))
    for c, doc in enumerate([3, 2, 1, 0]):
        rows = codes[off[doc]:off[doc] + lengths[doc]]
        want = sum(max(sum(int(T[i, m, r[m]]) for m in range(M)) for r in rows) for i in range(nq))
        assert got[c] == want


def test_pq_lut_scores_f16_table_brute_force():
    """An fp16 table is read exactly: the score equals the brute-force
    Python-float evaluation of sum_i max_j sum_m T[i][m][c] over the fp16
    values (m ascending, the oracle's order), and the same values given as
    fp64 (a misread half -- wrong byte order, exponent bias or subnormal --
    changes the score)."""
    g = np.random.default_rng(25)
    nq, M, K = 5, 16, 64
    T = (g.standard_normal((nq, M, K)) * 3).astype(np.float16)
    T[0, 0, :8] = np.array([6e-8, -6e-8, 1e-5, 65504, -65504, 0.0, -0.0, 2.0 ** -14], np.float16)
    lengths = np.array([1, 3, 9], np.int32)
    off = synth.offsets_of(lengths)
    codes = g.integers(0, K, size=(int(lengths.sum()), M)).astype(np.uint8)
    codes[0, 0] = 3   # the 65504 entry
    cand = np.array([2, 0, 1], np.int32)
    got = oracle.pq_lut_scores(T, codes, off, lengths, cand)
    np.testing.assert_array_equal(got, oracle.pq_lut_scores(T.astype(np.float64), codes, off, lengths, cand))
    for c, doc in enumerate(cand):
        rows = codes[off[doc]:off[doc] + lengths[doc]]
        total = 0.0
        for i in range(nq):
            best = -math.inf
            for r in rows:
                acc = 0.0
                for m in range(M):
                    acc += float(T[i, m, r[m]])
                best = max(best, acc)
            total += best
        assert got[c] == total


def test_pq_invalid_code_is_nan():
    cb = np.zeros((2, 4, 2), np.float32)
    codes = np.array([[0, 4]], np.uint8)
    got = oracle.pq_decompress_scores(np.ones((1, 4)), cb, codes, np.array([0]), np.array([1], np.int32),
                                      np.array([0], np.int32))
    assert math.isnan(got[0])


# ------------------------------------------------------------------- top-k

def _py_topk(scores, k):
    order = sorted(range(len(scores)),
                   key=lambda i: (1, 0.0, i) if math.isnan(scores[i]) else (0, -scores[i], i))
    out = [(scores[i], i) for i in order[:k]]
    out += [(-math.inf, -1)] * (k - len(out))
    return out


@pytest.mark.parametrize("seed", range(4))
def test_topk_matches_python_sort(seed):
    """Top-k equals Python's stable sort on (NaN last, score desc, pos asc),
    including ties, -inf, NaN and k > n."""
    g = np.random.default_rng(seed)
    n = int(g.integers(0, 300))
    s = np.round(g.standard_normal(n), 1)  # many ties
    s[g.random(n) < 0.05] = -np.inf
    s[g.random(n) < 0.05] = np.nan
    for k in (1, 10, 100, 400):
        got_s, got_p = oracle.topk(s, k)
        want = _py_topk(list(s), k)
        for (ws, wp), gs, gp in zip(want, got_s, got_p):
            assert gp == wp
            assert (math.isnan(ws) and math.isnan(gs)) or gs == ws


# --------------------------------------------------------------- FP8 E4M3

def test_e4m3_decode_exhaustive():
    """All 256 E4M3 patterns decode as torch's float8_e4m3fn -> float64."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    bits = np.arange(256, dtype=np.uint8)
    want = torch.from_numpy(bits.copy()).view(torch.float8_e4m3fn).double().numpy()
    got = np.array([oracle.e4m3_to_f64(int(b)) for b in bits])
    same = (got == want) | (np.isnan(got) & np.isnan(want))
    assert same.all()
    assert oracle.e4m3_to_f64(0x7E) == 448.0 and oracle.e4m3_to_f64(0x01) == 2.0 ** -9


def test_scaled_scores_match_explicit_dequantization():
    """Scaled-store scoring equals Eq. 1 on the explicitly dequantized fp64
    vectors (row scales for both the query and document tokens)."""
    g = np.random.default_rng(30)
    codes_t = g.integers(0, 256, size=(40, 16)).astype(np.uint8)
    codes_t[(codes_t & 0x7F) == 0x7F] = 0x11          # no NaN codes
    codes_q = g.integers(0, 256, size=(5, 16)).astype(np.uint8)
    codes_q[(codes_q & 0x7F) == 0x7F] = 0x22
    ts = g.uniform(0.01, 2.0, 40).astype(np.float32)
    qs = g.uniform(0.01, 2.0, 5).astype(np.float32)
    lengths = np.array([7, 0, 13, 20], np.int32)
    off = synth.offsets_of(lengths)
    cand = np.array([3, 1, 0, 2, 2], np.int32)
    got = oracle.dense_scores_scaled(codes_q, qs, codes_t, ts, off, lengths, cand,
                                     qdtype=oracle.E4M3, tdtype=oracle.E4M3)
    dec = np.vectorize(oracle.e4m3_to_f64)
    Xd = dec(codes_t) * ts[:, None].astype(np.float64)
    Qd = dec(codes_q) * qs[:, None].astype(np.float64)
    want = oracle.dense_scores(Qd, Xd, off, lengths, cand)
    assert np.array_equal(got, want)
    # and with unit scales it is the plain decode
    plain = oracle.dense_scores_scaled(Qd, None, Xd, None, off, lengths, cand)
    assert np.array_equal(plain, want)


def _torch_fp8():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    return torch


def test_e4m3_encode_matches_torch_cast_in_range():
    """Round to nearest even agrees with torch's float32 -> float8_e4m3fn
    cast on values below 464 (where torch does not overflow to NaN),
    including exact ties, subnormals and signed zeros."""
    torch = _torch_fp8()
    g = np.random.default_rng(31)
    mags = np.concatenate([g.uniform(0, 463.9, 3000), 2.0 ** g.uniform(-12, 8.85, 3000),
                           g.uniform(0, 2.0 ** -6, 500)])
    # every midpoint between adjacent finite codes is an exact tie
    vals = np.array([oracle.e4m3_to_f64(c) for c in range(127)])
    mids = (vals[:-1] + vals[1:]) / 2
    v = np.concatenate([mags, mids, [0.0, 448.0, 463.0]]).astype(np.float32)
    v = np.concatenate([v, -v])
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    got = np.array([oracle.e4m3_encode(x) for x in v], np.uint8)
    assert np.array_equal(got, want)


def test_e4m3_encode_saturates():
    for v, c in [(464.0, 0x7E), (480.0, 0x7E), (1e30, 0x7E), (-500.0, 0xFE), (448.5, 0x7E),
                 (2.0 ** -10, 0x00), (2.0 ** -10 + 2.0 ** -20, 0x01), (-(2.0 ** -11), 0x80)]:
        assert oracle.e4m3_encode(v) == c, v


@pytest.mark.parametrize("dt", ["f16", "bf16", "f32"])
def test_quantize_e4m3_rows(dt):
    """Per-row scale = amax / 448 in fp32, codes = cast(x / scale) (torch
    as the independent cast), the row maximum maps to +-448, a zero row has
    scale 0 and zero codes, and decode(code) * scale is within the E4M3
    rounding bound of x."""
    torch = _torch_fp8()
    from tests._common import oracle_view
    x = np.random.default_rng(32).standard_normal((64, 96)) * 0.1
    x[5] = 0
    x_in = synth.cast(x, dt)
    arr, code = oracle_view(x_in)
    codes, scales = oracle.quantize_e4m3(arr, dtype=code)
    xf = x_in.float()
    s_want = (xf.abs().amax(dim=1) / 448.0).numpy()
    assert np.array_equal(scales, s_want)
    assert scales[5] == 0 and not codes[5].any()
    nz = scales != 0
    q = (xf[nz] / torch.from_numpy(scales[nz])[:, None]).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(codes[nz], q)
    dec = np.vectorize(oracle.e4m3_to_f64)(codes).astype(np.float64) * scales[:, None]
    xd = xf.double().numpy()
    assert np.all(np.abs(np.abs(dec).max(axis=1)[nz] - np.abs(xd).max(axis=1)[nz]) <= 1e-6 * np.abs(xd).max())
    bound = np.maximum(np.abs(xd) * 2.0 ** -4, scales[:, None].astype(np.float64) * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(np.abs(dec - xd) <= bound)
