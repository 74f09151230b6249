"""The pair cache's record/check protocol (csrc/pair_cache.cu), restated on the CPU.

The cache may skip a pair only when its outcome is already known.  The model holds the
premises: a pair's decision (rotate or not) is a pure function of the contents of its two
blocks, and a rotation changes both blocks.  One simulation evaluates every pair of every step;
the other applies the kernel's protocol (block versions bumped on rotation, per-(step, slot)
records of (p, q, version p or -1, version q), a check that marks the slots whose record still
matches, a final record after the last step of a sweep).  Both must take the same decisions in
the same order, for several orderings, and the cached one must skip pairs once few rotate.
"""
import hashlib

import numpy as np
import pytest

from oracle import oracle


def h(*xs):
    return int.from_bytes(hashlib.blake2b(repr(xs).encode(), digest_size=8).digest(), "little")


def schedule(nb, ordering):
    if ordering == "round_robin":
        return [oracle.pairs_round_robin(nb, s) for s in range(nb - 1)]
    return [oracle.pairs_modulus(nb, k, modified=(ordering == "modulus_mod")) for k in range(nb)]


def decide(cp, cq, sweep_tol):
    # rotate iff the "off-diagonal" of the pair's contents is above the tolerance
    return (h(cp, cq) % 1000) < sweep_tol


def run(nb, ordering, sweeps, tols, cached_mode, seed):
    steps = schedule(nb, ordering)
    half = nb // 2
    content = [h(seed, b) for b in range(nb)]
    decisions, evaluated = [], 0
    # kernel state
    bver = [0] * nb
    pver = [[(-1, -1, -1, -1)] * half for _ in steps]
    cached = [1] * half
    skip = [1] * half
    for sw in range(sweeps):
        tol = tols[sw]
        for s, pairs in enumerate(steps):
            if cached_mode:
                # k_cache_step(rec = s - 1, chk = s): record the previous step, then check this one
                if s > 0:
                    record(steps, s - 1, cached, skip, bver, pver)
                for i, (p, q) in enumerate(pairs):
                    e = pver[s][i]
                    hit = e == (p, q, bver[p], bver[q])
                    cached[i] = 1 if hit else 0
                    if hit:
                        skip[i] = 1
            for i, (p, q) in enumerate(pairs):
                if cached_mode and cached[i]:
                    decisions.append((sw, s, i, False))
                    continue
                evaluated += 1
                rot = decide(content[p], content[q], tol)
                skip[i] = 0 if rot else 1
                decisions.append((sw, s, i, rot))
            for i, (p, q) in enumerate(pairs):  # the update: rotated pairs change both blocks
                if skip[i] == 0:
                    content[p], content[q] = h(content[p], content[q], 1), h(content[p], content[q], 2)
        if cached_mode:
            record(steps, len(steps) - 1, cached, skip, bver, pver)  # last step of the sweep
    return decisions, evaluated


def record(steps, r, cached, skip, bver, pver):
    for i, (p, q) in enumerate(steps[r]):
        if cached[i]:
            continue
        rot = skip[i] != 1
        if rot:
            bver[p] += 1
            bver[q] += 1
        pver[r][i] = (p, q, -1 if rot else bver[p], bver[q])


@pytest.mark.parametrize("ordering", ["round_robin", "modulus", "modulus_mod"])
@pytest.mark.parametrize("nb", [4, 8, 16, 30])
def test_cache_takes_the_same_decisions(ordering, nb):
    # a "tolerance" that makes most pairs rotate at first and few later; it only tightens, so a
    # decision not to rotate stays valid (the method's threshold is constant within a precision
    # phase, and the cache is reset when the phase changes)
    tols = [900, 600, 300, 100, 30, 10, 3, 1, 0, 0]
    ref, ev_ref = run(nb, ordering, len(tols), tols, False, seed=nb)
    got, ev_got = run(nb, ordering, len(tols), tols, True, seed=nb)
    rot_ref = [d for d in ref if d[3]]
    rot_got = [d for d in got if d[3]]
    assert rot_ref == rot_got
    assert ev_got < ev_ref
    # once nothing rotates for a whole sweep, the next sweep evaluates nothing at all
    last = [d for d in got if d[0] == len(tols) - 1]
    assert not any(d[3] for d in last)


# ---- the skip codes of one step with the fused FP32 step kernel (csrc/pivot.cu, capi.cu) ----
# per pair: 1 = no rotation (or a reported error), 2 = handed over to the FP64 pivot kernel,
# 0 = V_P formed for the separate update kernel, 3 = updated by the fused kernel itself.  The
# FP64 pivot kernel acts on 2 only (turning it into 0 on success, 1 on a singular block); the
# plain update acts on 0 only; the pair cache counts every code but 1 as a rotation.

def step_codes(outcomes, fused, fallback, fp64_ok):
    """outcomes[i] in {'none', 'rotate', 'handover'}: the FP32 pivot's result for pair i.
    Returns (updates applied per pair, final codes)."""
    code = [1 if o == "none" else (2 if o == "handover" else (3 if fused else 0)) for o in outcomes]
    applied = [1 if (fused and c == 3) else 0 for c in code]  # the fused kernel's own update
    if fallback:
        for i, c in enumerate(code):
            if c == 2:
                code[i] = 0 if fp64_ok[i] else 1
    for i, c in enumerate(code):  # the plain update kernel
        if c == 0:
            applied[i] += 1
    return applied, code


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("fallback", [False, True])
def test_fused_step_updates_each_pair_once(fused, fallback):
    import itertools

    kinds = ("none", "rotate", "handover")
    for outcomes in itertools.product(kinds, repeat=3):
        for fp64_ok in itertools.product((False, True), repeat=3):
            applied, code = step_codes(list(outcomes), fused, fallback, fp64_ok)
            for o, a, c, ok in zip(outcomes, applied, code, fp64_ok):
                if o == "rotate":
                    assert a == 1  # exactly once, by whichever kernel owns the pair
                elif o == "none":
                    assert a == 0 and c == 1
                else:  # handed over: rotated once by the FP64 path, or left for a later sweep
                    assert a == (1 if (fallback and ok) else 0)
                # the pair cache treats the pair as unchanged exactly when nothing was applied,
                # except a handover left unrotated (code 2), which it must re-evaluate
                rotated_for_cache = c != 1
                assert rotated_for_cache == (a == 1 or (o == "handover" and not fallback))
