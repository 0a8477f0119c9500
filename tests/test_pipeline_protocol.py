"""Discrete-event model of the stage ring of the tile pipeline (K4 matvec and
the K3 record pass), run on the CPU with random work assignments and
latencies.  It checks the protocol the kernel implements, not the kernel:

  * NS stages, one full and one empty barrier each (phase counters; a wait
    for phase P of parity p is exact only if the barrier is at P or P + 1);
  * the producer issues tile i into stage i % NS after the empty barrier
    completed the phase of tile i - NS, arrives there for the consumer warps
    tile i does not need (15 - need), then arms the full barrier and writes
    the stage's tile word seq[s] = i;
  * every consumer warp walks the tile list in order, computes the running
    first warp of each tile, skips the tiles it is not assigned to, and for
    its own tiles waits for seq[s] == i, then for the full barrier's phase,
    processes the stage and arrives on the empty barrier.

Checked: a consumer never reads a stage that holds another tile, every parity
wait sees the barrier at its phase or the next, every tile is processed by
exactly `need` warps, and the run ends (no deadlock)."""
import random

C = 15  # consumer warps


def _run(seed, ns, n_tiles=300, use_seq=True):
    rnd = random.Random(seed)
    need = [rnd.choice([1, 1, 2, 3, 5, 7, 15]) for _ in range(n_tiles)]
    full_phase = [0] * ns          # completed phases of the full barrier
    empty_phase = [0] * ns
    empty_cnt = [0] * ns
    seq = [-1] * ns
    holds = [None] * ns            # tile whose data is in the stage
    inflight = []                  # (landing time, stage, tile)
    issued = 0
    start = [0] * C
    nxt = [0] * C
    state = ["next"] * C
    busy = [0] * C
    cur = [None] * C
    done = [0] * n_tiles

    def arrive_empty(s, n):
        empty_cnt[s] += n
        assert empty_cnt[s] <= C
        if empty_cnt[s] == C:
            empty_cnt[s] = 0
            empty_phase[s] += 1

    t = 0
    while t < 200000:
        t += 1
        for x in list(inflight):
            if x[0] <= t:
                inflight.remove(x)
                holds[x[1]] = x[2]
                full_phase[x[1]] += 1
        if issued < n_tiles:
            s = issued % ns
            if (issued < ns or empty_phase[s] >= issued // ns) and rnd.random() < 0.5:
                arrive_empty(s, C - need[issued])
                inflight.append((t + rnd.randint(5, 60), s, issued))
                seq[s] = issued
                issued += 1
        for c in range(C):
            if busy[c] > t:
                continue
            if state[c] == "work":
                i = cur[c]
                s = i % ns
                assert holds[s] == i, ("stale stage", seed, c, i, holds[s])
                done[i] += 1
                arrive_empty(s, 1)
                state[c] = "next"
            if state[c] == "next":
                while nxt[c] < n_tiles:
                    i = nxt[c]
                    vcw = (c - start[c]) % C
                    start[c] = (start[c] + need[i]) % C
                    nxt[c] += 1
                    if vcw < need[i]:
                        cur[c] = i
                        state[c] = "seq"
                        break
                else:
                    state[c] = "end"
            if state[c] == "seq" and (seq[cur[c] % ns] == cur[c] or not use_seq):
                state[c] = "full"
            if state[c] == "full":
                i = cur[c]
                s = i % ns
                assert full_phase[s] in (i // ns, i // ns + 1), ("parity wait ambiguous", seed, i)
                if full_phase[s] == i // ns + 1:
                    state[c] = "work"
                    busy[c] = t + rnd.randint(1, 80)
        if issued == n_tiles and not inflight and all(x == "end" for x in state):
            break
    assert t < 200000, ("no progress", seed)
    assert done == need, ("tiles processed by the wrong number of warps", seed)


def test_stage_ring_protocol():
    for seed in range(150):
        _run(seed, ns=4 + seed % 3)


def test_skipping_without_the_tile_word_is_unsafe():
    """The same protocol without the seq wait: a warp that skipped tiles can
    meet its stage a phase early or late, which the model catches."""
    failures = 0
    for seed in range(60):
        try:
            _run(seed, ns=4 + seed % 3, use_seq=False)
        except AssertionError:
            failures += 1
    assert failures > 0
