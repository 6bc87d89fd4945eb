"""Planted mistakes in a copy of the oracle must each fail one of its pins.

Each mutant is a plausible slip (a swapped parameter, a sign, an index, a
dropped term, a wrong denominator, a wrong bit field, a wrong counter word)
applied to a temporary copy of ``oracle/zmc_oracle.c``; the committed source is
never modified.  The test shows the pins are strong enough that the oracle
cannot be wrong in any of these ways and still pass.
"""

import pytest

import oracle
from tests import oracle_pins as P

MUTANTS = {
    "harmonic_swap_ab": ("return p[0] * cos(phase) + p[1] * sin(phase);",
                         "return p[1] * cos(phase) + p[0] * sin(phase);"),
    "harmonic_sign": ("return p[0] * cos(phase) + p[1] * sin(phase);",
                      "return p[0] * cos(phase) - p[1] * sin(phase);"),
    "harmonic_k_index": ("phase += p[2 + i] * x[i];", "phase += p[1 + i] * x[i];"),
    "abslin_dropped_term": ("for (int i = 0; i < d; ++i)\n            s += p[1 + i] * x[i];",
                            "for (int i = 0; i < d - 1; ++i)\n            s += p[1 + i] * x[i];"),
    "gauss_missing_two": ("return p[0] * exp(-r2 / (2.0 * p[1] * p[1]));",
                          "return p[0] * exp(-r2 / (p[1] * p[1]));"),
    "poly_degree_off_by_one": ("for (int j = 0; j <= (int)f->deg; ++j)",
                               "for (int j = 0; j < (int)f->deg; ++j)"),
    "welford_m2": ("m2 += delta * (v - mean);", "m2 += delta * delta;"),
    "stderr_n_not_n_minus_1": ("stderr_out[j] = v * sqrt(m2 / (n * (n - 1.0)));",
                               "stderr_out[j] = v * sqrt(m2 / (n * n));"),
    "uniform_high_bits": ("return (double)(r & 0x7FFFFFu) * (1.0 / 8388608.0);",
                          "return (double)(r >> 9) * (1.0 / 8388608.0);"),
    "philox_weyl_swapped": ("k0 += ZO_PHILOX_W0;\n        k1 += ZO_PHILOX_W1;",
                            "k0 += ZO_PHILOX_W1;\n        k1 += ZO_PHILOX_W0;"),
    "philox_wrong_word": ("uint32_t n2 = hi0 ^ c[3] ^ k1;", "uint32_t n2 = hi0 ^ c[1] ^ k1;"),
    "counter_stream_word": (
        "uint32_t ctr[4] = {f->stream_id, (uint32_t)b, (uint32_t)(b >> 32), 0u};",
        "uint32_t ctr[4] = {0u, (uint32_t)b, (uint32_t)(b >> 32), f->stream_id};"),
    "counter_block_hi_dropped": (
        "uint32_t ctr[4] = {f->stream_id, (uint32_t)b, (uint32_t)(b >> 32), 0u};",
        "uint32_t ctr[4] = {f->stream_id, (uint32_t)b, 0u, 0u};"),
    "counter_words_swapped": (
        "uint32_t ctr[4] = {f->stream_id, (uint32_t)b, (uint32_t)(b >> 32), 0u};",
        "uint32_t ctr[4] = {(uint32_t)b, (uint32_t)(b >> 32), f->stream_id, 0u};"),
    "word_index": ("zo_field(f, s * (uint64_t)f->dim + i, cache)", "zo_field(f, s + i, cache)"),
    "fields_per_block_4": ("uint64_t b = c / 5;", "uint64_t b = c / 4;"),
    "field_stride_24": ("uint32_t first = 23u * (uint32_t)(c % 5);",
                        "uint32_t first = 24u * (uint32_t)(c % 5);"),
    "field_bit_order": ("r |= ((cache->words[q / 32] >> (q % 32)) & 1u) << j;",
                        "r |= ((cache->words[q / 32] >> (31 - q % 32)) & 1u) << j;"),
    "map_width": ("x[i] = f->lo[i] + (f->hi[i] - f->lo[i]) * zo_uniform(r);",
                  "x[i] = f->lo[i] + f->hi[i] * zo_uniform(r);"),
    "volume_missing": ("estimate[j] = v * mean;", "estimate[j] = mean;"),
}

# cheapest first; the first failing check ends a mutant's run
ORDER = ("special_cases", "philox_vs_independent", "word_layout", "bruteforce_small",
         "closed_forms", "stderr_calibration", "fig1", "eq2")


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, torch_philox):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new, 1))
    lib = oracle.compile_oracle(str(mutated), str(tmp_path / "libmutant.so"))
    orc = oracle.Oracle(lib)
    caught_by = None
    for check in ORDER:
        fn = getattr(P, check)
        try:
            if check in ("philox_vs_independent", "word_layout", "bruteforce_small"):
                fn(orc, torch_philox)
            else:
                fn(orc)
        except (AssertionError, ValueError, OverflowError):
            caught_by = check
            break
    assert caught_by is not None, f"mutant {name} passed every pin"
