"""Plant plausible mistakes in copies of the oracle; each must fail a pin.

Every mutant is a one-line edit of oracle/zmc_oracle.c (a dropped term, a
wrong sign, index or constant, a transposed operand), compiled on the CPU into
a temporary library.  The pins of oracle_pins.py then run against it, and at
least one of them must fail.  Nothing here touches the real oracle build.
"""
import os

import pytest

import oracle_pins as op
from oracle import oracle

MUTANTS = [
    ("philox multiplier", "#define ORC_PHILOX_M0 0xD2511F53u", "#define ORC_PHILOX_M0 0xD2511F55u"),
    ("philox key word", "uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c1 ^ k1;"),
    ("philox key bump", "if (round > 0) {", "if (round > 1) {"),
    ("philox rounds", "round < 10; ++round", "round < 9; ++round"),
    ("philox output order", "out[0] = c0; out[1] = c1;", "out[0] = c1; out[1] = c0;"),
    ("uniform odd term", "uint32_t odd = 2u * v + 1u;", "uint32_t odd = 2u * v;"),
    ("uniform scale", "return ldexp((double)odd, -24);", "return ldexp((double)odd, -23);"),
    ("word call index", "oracle_call(seed, p, t, w >> 2, out);", "oracle_call(seed, p, t, w >> 1, out);"),
    ("field call index", "uint64_t j = i / 5u;", "uint64_t j = i / 4u;"),
    ("field slot", "int m = (int)(i % 5u);", "int m = (int)(i % 4u);"),
    ("field width", "int bit = 23 * m;", "int bit = 24 * m;"),
    ("field mask", "return (uint32_t)((pair >> sh) & 0x7fffffu);", "return (uint32_t)((pair >> sh) & 0x3fffffu);"),
    ("field word order", "uint64_t pair = (uint64_t)out[q] | ((uint64_t)out[q + 1] << 32);",
     "uint64_t pair = (uint64_t)out[q + 1] | ((uint64_t)out[q] << 32);"),
    ("trial word", "ctr[1] = (uint32_t)t;", "ctr[1] = (uint32_t)(t + 1);"),
    ("point high word", "ctr[3] = (uint32_t)((uint64_t)p >> 32);", "ctr[3] = 0u;"),
    ("lane of the call", "return out[w & 3u];", "return out[(w + 1) & 3u];"),
    ("field of a sample", "uint64_t i = (uint64_t)s * (uint64_t)N + (uint64_t)k;",
     "uint64_t i = (uint64_t)s * 4u + (uint64_t)k;"),
    ("box base", "y[k] = fma(hi[k] - lo[k], u, lo[k]);", "y[k] = fma(hi[k] - lo[k], u, hi[k]);"),
    ("box width", "y[k] = fma(hi[k] - lo[k], u, lo[k]);", "y[k] = fma(hi[k], u, lo[k]);"),
    ("decode order", "for (int i = M - 1; i >= 0; --i) {", "for (int i = 0; i < M; ++i) {"),
    ("list offset", "x[i] = vals[offset + digit[i]];", "x[i] = vals[digit[i]];"),
    ("cosprod transposed", "g *= cos(x[k] * y[k]);", "g *= cos(x[N - 1 - k] * y[k]);"),
    ("gauss sigma squared", "return exp(-q / (2.0 * sigma * sigma));", "return exp(-q / (2.0 * sigma));"),
    ("gauss centre", "q += (y[k] - x[k]) * (y[k] - x[k]);", "q += (y[k] + x[k]) * (y[k] + x[k]);"),
    ("poly square", "g *= 1.0 + x[k] * y[k] * y[k];", "g *= 1.0 + x[k] * y[k];"),
    ("osc sign", "return cos(lin + 0.1 * quad);", "return cos(lin - 0.1 * quad);"),
    ("sinsum parameter sum", "for (int l = 0; l < M; ++l) a += x[l];", "for (int l = 1; l < M; ++l) a += x[l];"),
    ("volume term", "for (int k = 0; k < N; ++k) V *= hi[k] - lo[k];",
     "for (int k = 1; k < N; ++k) V *= hi[k] - lo[k];"),
    ("estimate divisor", "I[t] = V * s1 / (double)S;", "I[t] = V * s1 / (double)(S - 1);"),
    ("square sum", "s2 += g * g;", "s2 += g;"),
    ("mean drops a trial", "for (int t = 0; t < T; ++t) sum += I[t];", "for (int t = 1; t < T; ++t) sum += I[t];"),
    ("stderr divisor", "sqrt(dev2 / ((double)T * (double)(T - 1)))", "sqrt(dev2 / ((double)T * (double)T))"),
    ("stderr square", "dev2 += (I[t] - mean) * (I[t] - mean);", "dev2 += fabs(I[t] - mean);"),
    ("pooled variance divisor", "/ (double)(S - 1);", "/ (double)S;"),
    ("pooled stderr volume", "errw = V * sqrt(pooled_var / ((double)T * (double)S));",
     "errw = sqrt(pooled_var / ((double)T * (double)S));"),
]


@pytest.mark.parametrize("name,before,after", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_fails_a_pin(tmp_path, philox_ref, name, before, after):
    src = open(oracle.SOURCE).read()
    assert src.count(before) == 1, "mutation site must be unique: " + before
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(before, after))
    lib = oracle.compile_source(str(mutated), str(tmp_path / "libmutant.so"))
    O = oracle.Oracle(lib)
    with pytest.raises((AssertionError, ValueError)):
        op.all_pins(O, philox_ref, fast=True)
