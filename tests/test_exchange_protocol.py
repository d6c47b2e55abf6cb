"""The pivot exchange of the CTA-group pivoted QR (qrcp_grid_kernel), modelled
on the host.

Every CTA of a matrix runs, for steps i = 0, 1, ...: write its proposal and
reflector into buffer i % 2; add one to that buffer's arrival counter; wait
until the counter reaches G * (i // 2 + 1); read every CTA's buffer-(i % 2)
entry.  The kernel relies on two facts, checked here over many random
interleavings of G CTAs (one action of one CTA at a time):

* every read of step i sees step i's entry of every CTA (no CTA can rewrite a
  buffer before all CTAs have read it: rewriting it is step i + 2, which needs
  every CTA's step-(i + 1) arrival, which follows its step-i reads);
* the waits always end (no deadlock) and all CTAs leave after the same step.

A single buffer (the same protocol with buffer 0 for every step) must fail
the first check, which shows that the check can fail.
"""
import random

import pytest


def _run(G, steps, buffers, seed):
    rng = random.Random(seed)
    slot = [[None] * G for _ in range(buffers)]
    count = [0] * buffers
    # per CTA: (step, phase) with phases 0 write, 1 arrive, 2 wait, 3 read
    state = [[0, 0] for _ in range(G)]
    stale = 0
    while any(s[0] < steps for s in state):
        runnable = []
        for r, (i, ph) in enumerate(state):
            if i >= steps:
                continue
            b = i % buffers
            if ph == 2 and count[b] < G * (i // buffers + 1):
                continue  # still waiting
            runnable.append(r)
        assert runnable, "deadlock"
        r = rng.choice(runnable)
        i, ph = state[r]
        b = i % buffers
        if ph == 0:
            slot[b][r] = i
        elif ph == 1:
            count[b] += 1
        elif ph == 3:
            stale += sum(1 for q in range(G) if slot[b][q] != i)
        state[r] = [i + 1, 0] if ph == 3 else [i, ph + 1]
    return stale


@pytest.mark.parametrize("G", [2, 3, 17, 40])
def test_two_buffers_never_read_a_rewritten_slot(G):
    for seed in range(60):
        assert _run(G, 9, 2, seed) == 0


def test_one_buffer_would_be_overwritten():
    assert sum(_run(17, 9, 1, seed) for seed in range(60)) > 0
