"""The stage protocol of the stored-matrix streaming kernel, checked as a
model under random schedules (no GPU).

One producer copies chunks 0, 1, ... into a ring of S stages (chunk q goes
to stage q mod S after the consumer of chunk q - S freed that stage); work
items of one or more chunks are dealt round-robin to consumer warps, so a
warp waits for stages that other warps used before it.  An mbarrier parity
wait only distinguishes the current phase from the one before it: waiting
for parity P returns at once when the phase just completed has parity P.
A consumer that waits for round r of a stage while round r - 1 is still in
flight would therefore pass early.  The kernel prevents this by first
waiting until the producer has issued its chunk (the producer issues round
r only after round r - 1 was consumed).  The model shows both: without the
issue gate consumers read stages before their chunk landed; with it, every
read sees its own chunk and no schedule deadlocks.
"""
import random


def _parity_done(completed_phases, parity):
    # try_wait.parity(P): true iff the phase just completed has parity P
    return (completed_phases & 1) != parity


def _run(item_chunks, stages, warps, gate, seed):
    rnd = random.Random(seed)
    full_done = [0] * stages
    empty_done = [0] * stages
    landed = [None] * stages
    inflight = []
    issued = 0
    seq0, s = [], 0
    for c in item_chunks:
        seq0.append(s)
        s += c
    nq = s
    queues = []
    for w in range(warps):
        q = []
        for it in range(w, len(item_chunks), warps):
            q += [seq0[it] + p for p in range(item_chunks[it])]
        queues.append(q)
    pos = [0] * warps
    bad_reads = 0
    for _ in range(200000):
        actors = (["P"] if issued < nq else []) + (["T"] if inflight else [])
        actors += [w for w in range(warps) if pos[w] < len(queues[w])]
        if not actors:
            return "ok", bad_reads
        a = rnd.choice(actors)
        if a == "P":
            k = issued % stages
            if issued >= stages and not _parity_done(empty_done[k], (issued // stages - 1) & 1):
                continue
            inflight.append((k, issued))
            issued += 1
        elif a == "T":
            k, q = inflight.pop(rnd.randrange(len(inflight)))
            landed[k] = q
            full_done[k] += 1
        else:
            q = queues[a][pos[a]]
            k = q % stages
            if gate and not issued > q:
                continue
            if not _parity_done(full_done[k], (q // stages) & 1):
                continue
            if landed[k] != q:
                bad_reads += 1
            empty_done[k] += 1
            pos[a] += 1
    return "stuck", bad_reads


def _cases(n):
    for seed in range(n):
        rnd = random.Random(seed)
        items = [rnd.choice([1, 1, 2, 3]) for _ in range(rnd.randint(1, 50))]
        yield items, rnd.choice([2, 3, 6, 9]), rnd.choice([4, 8]), seed


def test_issue_gate_makes_every_read_see_its_chunk():
    for items, stages, warps, seed in _cases(150):
        state, bad = _run(items, stages, warps, gate=True, seed=seed)
        assert state == "ok" and bad == 0, (items, stages, warps, seed, state, bad)


def test_without_the_gate_parity_waits_pass_early():
    failures = sum(_run(items, stages, warps, gate=False, seed=seed) != ("ok", 0)
                   for items, stages, warps, seed in _cases(60))
    assert failures > 0
