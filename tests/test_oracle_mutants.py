"""Strength of the oracle's pins.  Each plausible mistake below is planted in
a copy of the oracle's C source (a transposed index, a swapped class column,
a dropped or sign-flipped entropy term, a wrong log argument, a reversed
tie-break, a repeated or skipped SNP, a broken top-N list, an off-by-one
count, a loosened check); the copy
is compiled into a temporary directory and the pin tests run against it in a
child process (FC_ORACLE_LIB).  Every mutant must fail them (a failing
assertion, not a crash), and the unmodified source, compiled the same way,
must pass."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "cell index transposed": (
        "cell = cell * 3 + G[(int64_t)combo[t] * M + m];",
        "cell = cell * 3 + G[(int64_t)combo[k - 1 - t] * M + m];"),
    "case and control columns swapped": (
        "int col = ph[m] == 1 ? 0 : 1;",
        "int col = ph[m] == 1 ? 1 : 0;"),
    "H(Y) dropped": (
        "return hx + hy - hxy;",
        "return hx - hxy;"),
    "joint entropy sign flipped": (
        "if (nxy > 0.0) hxy -= (nxy / N) * log(nxy / N);",
        "if (nxy > 0.0) hxy += (nxy / N) * log(nxy / N);"),
    "log of a count instead of a probability": (
        "if (nx > 0.0) hx -= (nx / N) * log(nx / N);",
        "if (nx > 0.0) hx -= (nx / N) * log(nx);"),
    "tie-break reversed": (
        "if (a->idx[t] != b->idx[t]) return a->idx[t] < b->idx[t];",
        "if (a->idx[t] != b->idx[t]) return a->idx[t] > b->idx[t];"),
    "extension repeats the last prefix SNP": (
        "int64_t j0 = plen == 0 ? 0 : (int64_t)pfx[plen - 1] + 1;",
        "int64_t j0 = plen == 0 ? 0 : (int64_t)pfx[plen - 1];"),
    "extension skips the first candidate": (
        "int64_t j0 = plen == 0 ? 0 : (int64_t)pfx[plen - 1] + 1;",
        "int64_t j0 = plen == 0 ? 1 : (int64_t)pfx[plen - 1] + 2;"),
    "distribution counts one extension too many": (
        "counts[ordinal % p] += (uint64_t)(n - 1 - (int64_t)pfx[plen - 1]);",
        "counts[ordinal % p] += (uint64_t)(n - (int64_t)pfx[plen - 1]);"),
    "distribution deals prefixes to the wrong unit": (
        "counts[ordinal % p] +=",
        "counts[(ordinal + 1) % p] +="),
    "full list evicts its best entry": (
        "memmove(&L->list[0], &L->list[1], sizeof(orc_entry) * (size_t)(L->size - 1));",
        ";"),
    "full list never takes a better entry": (
        "if (L->size < L->cap || ranks_above(e, &L->list[0], L->k)) {",
        "if (L->size < L->cap) {"),
    "binomial coefficient off by one": (
        "acc = acc * (unsigned __int128)(n - r + i) / (unsigned __int128)i;",
        "acc = acc * (unsigned __int128)(n - r + i + 1) / (unsigned __int128)i;"),
    "genotype 3 accepted": (
        "if (G[i] > 2) return ORC_EINVAL;",
        "if (G[i] > 3) return ORC_EINVAL;"),
}


def _compile(tmp, name, text):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", lib, src, "-lm"])
    return lib


def _run_pins(lib):
    """pytest's exit status over the pin tests with `lib` as the oracle: 0
    all passed, 1 some failed (anything else: a crash or an error)."""
    env = dict(os.environ, FC_ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-400:]


def test_every_planted_mistake_fails_the_pins(tmp_path):
    text = open(SRC).read()
    libs = {"unmodified": _compile(str(tmp_path), "unmodified", text)}
    for n, (name, (old, new)) in enumerate(MUTANTS.items()):
        assert text.count(old) == 1, name    # each mutation site exists exactly once
        libs[name] = _compile(str(tmp_path), f"mutant{n}", text.replace(old, new))
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = dict(zip(libs, ex.map(_run_pins, libs.values())))
    rc, out = results.pop("unmodified")
    assert rc == 0, out
    # Caught by a failing pin, not by a crash.
    wrong = {name: rc for name, (rc, _) in results.items() if rc != 1}
    assert not wrong, wrong
