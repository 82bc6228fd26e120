"""CPU checks of the kernels' integer arithmetic (csrc/arith.h compiled for the host).

The header is shared by host and device code, so compiling it with g++ tests
the same expressions the kernels evaluate: the division by a precomputed
reciprocal, the Jaccard and Dice required overlaps, and Cosine's exact
ceil(t sqrt(|r||s|)).
"""
import math
import os
import random
import subprocess

import pytest

from conftest import ROOT

HARNESS = r'''
#include <cstdio>
#include <cstdint>
#include "arith.h"
int main() {
    char kind;
    while (scanf(" %c", &kind) == 1) {
        if (kind == 'd') {
            unsigned long long x, d;
            if (scanf("%llu %llu", &x, &d) != 2) return 2;
            printf("%llu\n", (unsigned long long)ssj::div_by_magic(x, d, ssj::div_magic(d)));
        } else if (kind == 'c') {
            unsigned nr, ns, p, q;
            if (scanf("%u %u %u %u", &nr, &ns, &p, &q) != 4) return 2;
            printf("%u\n", ssj::required_overlap_cosine(p, q, nr, ns));
        } else if (kind == 'e') {
            unsigned nr, ns, p, q;
            if (scanf("%u %u %u %u", &nr, &ns, &p, &q) != 4) return 2;
            printf("%u\n", ssj::required_overlap_magic(nr, ns, p, 2 * q, ssj::div_magic(2ull * q)));
        } else {
            unsigned nr, ns, p, q;
            if (scanf("%u %u %u %u", &nr, &ns, &p, &q) != 4) return 2;
            printf("%u\n", ssj::required_overlap_magic(nr, ns, p, p + q, ssj::div_magic((uint64_t)p + q)));
        }
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("arith")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_1812_09141_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    return str(exe)


def _run(exe, lines):
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
    return [int(x) for x in out.stdout.split()]


def test_division_by_reciprocal_is_exact(harness):
    rng = random.Random(1)
    cases = []
    for d in [2, 3, 5, 7, 9, 10, 20, 39, 2**31 - 1, 2**32 - 1, 2**32 + 1, 2**63 - 1]:
        for x in [0, 1, d - 1, d, d + 1, 2**63 - 1, 2**64 - 1, 2**64 - d, (2**64 - 1) // d * d]:
            cases.append((x % 2**64, d))
    for _ in range(20000):
        d = rng.choice([rng.randint(2, 100), rng.randint(2, 2**32), rng.randint(2, 2**64 - 1)])
        x = rng.choice([rng.randint(0, 2**64 - 1), rng.randint(0, 2**40), rng.randint(0, 1000) * d + rng.randint(0, d - 1)]) % 2**64
        cases.append((x, d))
    got = _run(harness, [f"d {x} {d}" for x, d in cases])
    assert got == [x // d for x, d in cases]


def test_required_overlap_matches_exact_ceiling(harness):
    rng = random.Random(2)
    cases = [(nr, ns, p, q) for p, q in [(19, 20), (9, 10), (4, 5), (3, 5), (1, 1), (1, 2)]
             for nr in range(0, 60) for ns in range(0, 60)]
    for _ in range(20000):
        p = rng.randint(1, 2**31 - 1)
        q = rng.randint(p, 2**31 - 1)
        cases.append((rng.randint(0, 2**31 - 1), rng.randint(0, 2**31 - 1), p, q))
    got = _run(harness, [f"r {nr} {ns} {p} {q}" for nr, ns, p, q in cases])
    assert got == [-(-p * (nr + ns) // (p + q)) for nr, ns, p, q in cases]


def _cosine_exact(nr, ns, p, q):
    """Least o with (q o)^2 >= p^2 nr ns, capped at min(nr, ns) + 1; never for an empty set."""
    if nr == 0 or ns == 0:
        return 0xFFFFFFFF
    x = p * p * nr * ns
    y = math.isqrt(x)
    if y * y < x:
        y += 1
    return min(-(-y // q), min(nr, ns) + 1)


def test_cosine_required_overlap_is_exact(harness):
    rng = random.Random(3)
    cases = [(nr, ns, p, q) for p, q in [(19, 20), (9, 10), (4, 5), (3, 5), (1, 1), (1, 2), (1, 3)]
             for nr in range(0, 50) for ns in range(0, 50)]
    for _ in range(20000):
        p = rng.randint(1, 2**31 - 1)
        q = rng.randint(p, 2**31 - 1)
        big = rng.random() < 0.5
        nr = rng.randint(0, 2**32 - 1) if big else rng.randint(0, 5000)
        ns = rng.randint(0, 2**32 - 1) if big else rng.randint(0, 5000)
        cases.append((nr, ns, p, q))
    # perfect squares: ties decided exactly
    for k in range(1, 200):
        cases.append((k * k, 4 * k * k, 1, 2))
        cases.append((9 * k, k, 2, 3))
    got = _run(harness, [f"c {nr} {ns} {p} {q}" for nr, ns, p, q in cases])
    assert got == [_cosine_exact(*c) for c in cases]


def test_dice_required_overlap_matches_exact_ceiling(harness):
    rng = random.Random(4)
    cases = [(nr, ns, p, q) for p, q in [(19, 20), (4, 5), (3, 5), (1, 1), (1, 2)]
             for nr in range(0, 40) for ns in range(0, 40)]
    for _ in range(20000):
        p = rng.randint(1, 2**31 - 1)
        q = rng.randint(p, 2**31 - 1)
        cases.append((rng.randint(0, 2**31 - 1), rng.randint(0, 2**31 - 1), p, q))
    got = _run(harness, [f"e {nr} {ns} {p} {q}" for nr, ns, p, q in cases])
    assert got == [-(-p * (nr + ns) // (2 * q)) for nr, ns, p, q in cases]
