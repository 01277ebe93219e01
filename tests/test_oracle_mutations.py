"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle/isg_oracle.c, builds it, binds
the wrapper to it and runs the pins of tests/test_oracle_pins.py: at least one
pin must fail.  Only the oracle is mutated, only on the CPU."""
import os
import shutil
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "isg_oracle.c")

MUTANTS = {
    "wrong -x coupling": ("Jb[1] = Jx[idx(L, xm, y, z)];", "Jb[1] = Jx[i];"),
    "wrong -z neighbour": ("nb[5] = s[idx(L, x, y, zm)];", "nb[5] = s[idx(L, x, y, zp)];"),
    "counts satisfied bonds": ("if (J[k] * s * nb[k] == -1) ++u;", "if (J[k] * s * nb[k] == 1) ++u;"),
    "<= instead of <": ("return d < thr[dE / 4];", "return d <= thr[dE / 4];"),
    "threshold factor": ("exp(-4.0 * (double)k * beta)", "exp(-2.0 * (double)k * beta)"),
    "threshold index": ("return d < thr[dE / 4];", "return d < thr[4 - dE / 4];"),
    "MINSTD multiplier": ("(uint64_t)16807u * (uint64_t)(*x)", "(uint64_t)16806u * (uint64_t)(*x)"),
    "MINSTD draw not doubled": ("return minstd_next(&st->minstd) << 1;", "return minstd_next(&st->minstd);"),
    "MT19937 tempering": ("v ^= (v << 15) & 0xEFC60000u;", "v ^= (v << 15) & 0xEFC40000u;"),
    "MT19937 seeding": ("1812433253u * (m->x[k - 1] ^ (m->x[k - 1] >> 30))",
                        "1812433253u * (m->x[k - 1] ^ (m->x[k - 1] >> 29))"),
    "draw skipped for downhill moves": ("            uint32_t d = stream_draw(&o->st[t]);\n"
                                        "            int u = or_unsatisfied(s[i], nb, Jb);",
                                        "            int u = or_unsatisfied(s[i], nb, Jb);\n"
                                        "            uint32_t d = u < 3 ? stream_draw(&o->st[t]) : 0u;"),
    "energy change sign": ("dE += 12 - 4 * u;", "dE += 4 * u - 12;"),
    "energy sign": ("E -= o->J[i] * o->s[i]", "E += o->J[i] * o->s[i]"),
    "energy misses z bonds": ("                E -= o->J[2 * N + i] * o->s[i] * o->s[idx(L, x, y, (z + 1) % L)];\n", ""),
    "coupling bias": ("(or_splitmix64(seed_J ^ SALT_COUPLINGS, 3 * (uint64_t)i + (uint64_t)d) >> 63) ? -1 : 1",
                      "(or_splitmix64(seed_J ^ SALT_COUPLINGS, 3 * (uint64_t)i + (uint64_t)d) >> 62) ? -1 : 1"),
    "splitmix increment": ("(n + 1u) * 0x9E3779B97F4A7C15ull", "n * 0x9E3779B97F4A7C15ull"),
    "overlap sign": ("q += a->s[i] * b->s[i];", "q -= a->s[i] * b->s[i];"),
    "hash keys": ("if (o->s[i] == 1) h ^= or_splitmix64(SALT_HASH, (uint64_t)i);",
                  "if (o->s[i] == 1) h ^= or_splitmix64(SALT_HASH, (uint64_t)i + 1);"),
    "stream rows": ("if (s > 8192) s = 8192;", "if (s > 4096) s = 4096;"),
    "Parisi-Rapuano short lag": ("p->w[(k + 61 - 24) % 61]", "p->w[(k + 61 - 23) % 61]"),
    "Parisi-Rapuano output lag": ("uint32_t lag61 = p->w[k];", "uint32_t lag61 = p->w[(k + 1) % 61];"),
    "Parisi-Rapuano xor for add": ("uint32_t v = lag24 + lag55;", "uint32_t v = lag24 ^ lag55;"),
    "Parisi-Rapuano seeding": ("p->w[j] = (uint32_t)(or_splitmix64(v, (uint64_t)j) >> 32);",
                               "p->w[j] = (uint32_t)or_splitmix64(v, (uint64_t)j);"),
}

# pins that need no tmp_path fixture, with their parameters
PIN_CALLS = [
    (pins.test_generator_golden_values, {}),
    (pins.test_mt19937_matches_numpy_legacy_seeding, {"seed": 12345}),
    (pins.test_thresholds_golden_and_limits, {}),
    (pins.test_stencil_exhaustive_energy_change, {}),
    (pins.test_energy_closed_forms, {"L": 4}),
    (pins.test_energy_symmetries, {"L": 4}),
    (pins.test_tracked_energy_equals_scratch, {"L": 6, "beta": 1 / 1.1, "kind": 1}),
    (pins.test_tracked_energy_equals_scratch, {"L": 4, "beta": 0.3, "kind": 0}),
    (pins.test_zero_temperature_energy_nonincreasing, {"kind": 1}),
    (pins.test_gauge_transform_maps_trajectory, {"L": 8, "kind": 0}),
    (pins.test_acceptance_frequency_in_sweeps, {"kind": 0}),
    (pins.test_acceptance_frequency_in_sweeps, {"kind": 1}),
    (pins.test_equilibrium_energy_T5, {"kind": 1}),
    (pins.test_overlap_and_hash_properties, {}),
    (pins.test_stream_partition_and_draw_counts, {}),
    (pins.test_coupling_and_spin_balance, {}),
    (pins.test_parisi_rapuano_companion_matrix_powers, {"v": 77}),
    (pins.test_parisi_rapuano_low_bits_polynomial_jump, {}),
]


def _build_mutant(tmp, name, old, new):
    src = open(SRC).read()
    assert old in src, "mutation no longer applies: %s" % name
    d = tmp / name.replace(" ", "_").replace("<", "lt").replace("=", "eq").replace("/", "_")
    d.mkdir()
    shutil.copy(os.path.join(os.path.dirname(SRC), "isg_oracle.h"), d / "isg_oracle.h")
    (d / "isg_oracle.c").write_text(src.replace(old, new, 1))
    so = d / "libmut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", str(so),
                    str(d / "isg_oracle.c"), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, name, old, new)
    caught = []
    oracle.use_library(so)
    try:
        for fn, kw in PIN_CALLS:
            try:
                fn(**kw)
            except (AssertionError, ValueError):
                caught.append(fn.__name__)
                break
    finally:
        oracle.use_library(None)
    assert caught, "no pin caught the planted mistake '%s'" % name


def test_unmutated_copy_passes_every_pin(tmp_path):
    so = _build_mutant(tmp_path, "identity", "#include <math.h>", "#include <math.h>")
    oracle.use_library(so)
    try:
        for fn, kw in PIN_CALLS:
            fn(**kw)
    finally:
        oracle.use_library(None)
