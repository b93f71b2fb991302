"""Model check of the copy/barrier protocol of the staged persistent passes.

The staged row pass (``csrc/krs.cuh``) and column pass (``csrc/kcs.cuh``)
give one CTA two thread groups and one staging buffer. The CTA's tiles are
i = 0, 1, 2, ...; tile i belongs to group i mod 2, whose k-th tile
(k = i div 2) completes phase k of its mbarrier. Tile 0's copy is started
before the loop; the group holding tile i starts the copy of tile i + 1
into the stage once all of its threads have read tile i from it. The
column pass also copies each tile's node constants into slot i mod 4 of a
four-slot ring, read again in the tile's epilogue.

A group waits with ``mbarrier.try_wait.parity(k & 1)``, which returns true
when the barrier's completed-phase count c has the other parity. That is
the same as "phase k has completed" only while c is k or k + 1. This model
lets a random scheduler interleave the two groups and the copy engine, and
asserts that:

* every wait that returns sees c in {k, k + 1};
* when a group reads the stage, the stage holds its tile and no copy into
  the stage is in flight;
* a copy is never started into the stage while another one is in flight;
* a node-constant slot is never overwritten before its tile's epilogue;
* the row pass's bounded drain at exit (the parity wait for the last copy
  a thread started) finds exactly that copy's phase completed, so it cannot
  alias a later one (the column pass drains with cp.async.wait_all).

It checks the protocol the kernels implement, not the kernels themselves.
It also plants two mistakes: a copy started before the stage is read, and
a two-slot node ring. The model must catch both.
"""
import random

import pytest


class ProtocolError(AssertionError):
    pass


def run(n_tiles, seed, *, late_fetch=False, slots=4, fetch_before_read=False, max_steps=100000):
    """One randomly scheduled run of the staged protocol for one CTA with
    n_tiles tiles; raises ProtocolError on a violated invariant."""
    rng = random.Random(seed)
    completed = [0, 0]          # completed phases of mbarrier 0, 1
    stage = None                # tile whose data the stage holds
    in_flight = None            # tile being copied into the stage
    slot = [None] * slots       # node-constant ring: which tile's constants each slot holds
    last_copy = {0: None, 1: None}  # last tile whose copy each group started (drain)
    last_copy[0] = 0 if n_tiles > 0 else None  # tile 0 is started before the loop
    if n_tiles > 0:
        in_flight = 0

    # per-group program: states "wait", "read", "hook", "epilogue", "done"
    pc = {g: ("wait", g) if g < n_tiles else ("done", None) for g in (0, 1)}

    def start_copy(tile, by):
        nonlocal in_flight
        if in_flight is not None:
            raise ProtocolError(f"copy of tile {tile} started while tile {in_flight} is in flight")
        in_flight = tile
        last_copy[by] = tile

    def wait_ok(g, k):
        c = completed[g]
        passes = (c & 1) != (k & 1)
        if passes and c not in (k, k + 1):
            raise ProtocolError(f"group {g} waits for phase {k} and passes with {c} completed phases")
        return passes

    steps = 0
    while any(pc[g][0] != "done" for g in (0, 1)) or in_flight is not None:
        steps += 1
        if steps > max_steps:
            raise ProtocolError("no progress (deadlock)")
        actors = [g for g in (0, 1) if pc[g][0] != "done"]
        if in_flight is not None:
            actors.append("copy")
        a = rng.choice(actors)
        if a == "copy":
            # the copy lands: the stage and the slot take the tile, the barrier completes a phase
            t = in_flight
            in_flight = None
            stage = t
            s = t % slots
            if slot[s] is not None and slot[s][1] != "used":
                raise ProtocolError(f"slot {s} overwritten by tile {t} before tile {slot[s][0]}'s epilogue")
            slot[s] = (t, "fresh")
            completed[t % 2] += 1
            continue
        g = a
        state, i = pc[g]
        k = i // 2
        if state == "wait":
            if fetch_before_read and i + 1 < n_tiles and last_copy[g] != i + 1 and in_flight is None:
                start_copy(i + 1, g)  # planted mistake: the next copy before this tile is read
            if wait_ok(g, k):
                pc[g] = ("read", i)
        elif state == "read":
            if stage != i or in_flight is not None:
                raise ProtocolError(f"group {g} reads tile {i} while the stage holds {stage}, in flight {in_flight}")
            if slot[i % slots] is None or slot[i % slots][0] != i:
                raise ProtocolError(f"tile {i}'s node constants are not in slot {i % slots}")
            pc[g] = ("hook", i)
        elif state == "hook":
            # all threads of the group have read tile i (named barrier); with late_fetch
            # the copy starts after the first transform pass, otherwise at once
            if late_fetch and rng.random() < 0.5:
                continue
            if i + 1 < n_tiles and last_copy[g] != i + 1:
                start_copy(i + 1, g)
            pc[g] = ("epilogue", i)
        elif state == "epilogue":
            if slot[i % slots] is None or slot[i % slots][0] != i:
                raise ProtocolError(f"tile {i}'s node constants were overwritten before its epilogue")
            slot[i % slots] = (i, "used")
            nxt = i + 2
            pc[g] = ("wait", nxt) if nxt < n_tiles else ("done", None)
    # drain: each group waits for the last copy it started (phase kb of its barrier)
    for g in (0, 1):
        t = last_copy[g]
        if t is None:
            continue
        gb, kb = t % 2, t // 2
        c = completed[gb]
        if c not in (kb + 1,):  # the copy landed; a later phase would alias the parity wait
            raise ProtocolError(f"drain of tile {t}: barrier {gb} has {c} completed phases, expected {kb + 1}")
    return steps


@pytest.mark.parametrize("late_fetch", [False, True])
@pytest.mark.parametrize("n_tiles", [0, 1, 2, 3, 4, 7, 16])
def test_staged_protocol_invariants(n_tiles, late_fetch):
    for seed in range(1000):
        run(n_tiles, seed, late_fetch=late_fetch)


def test_model_catches_a_copy_started_before_the_stage_is_read():
    with pytest.raises(ProtocolError):
        for seed in range(300):
            run(8, seed, fetch_before_read=True)


def test_model_catches_a_two_slot_node_ring():
    with pytest.raises(ProtocolError):
        for seed in range(300):
            run(8, seed, slots=2)
