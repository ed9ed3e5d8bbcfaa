"""Host-side ordering of the ensemble's shared launches (csrc/ps_worklist.h),
compiled alone with the host C++ compiler and run on generated ensembles.

The persistent launch hands out tickets in list order and a CTA waits, before
its first tile of a pass instance, for the member's previous pass instance to
be complete.  That is deadlock-free only if every dependency owns lower
tickets; the queue simulation below checks it for any number of CTAs, and
checks itself on a list that breaks the rule.
"""

import math
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1808_01309_gb300", "csrc")

# pass kinds in a member's sequence (the energy sum only after the first
# z-inverse of the last step, and nothing waits for it)
ZINV, SUM, YINV, XPASS, YFWD, ZFWD, UPDATE = range(7)


@pytest.fixture(scope="module")
def worklist_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("wl") / "worklist_main")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "worklist_main.cpp"), "-o", exe], check=True)
    return exe


def member_sequence(rng, nsteps, stages):
    """(kind, ntiles, per, chain) of one member's pass instances in order."""
    seq = []
    for s in range(nsteps):
        for st in range(stages):
            for kind in (ZINV, SUM, YINV, XPASS, YFWD, ZFWD, UPDATE):
                if kind == SUM and not (s == nsteps - 1 and st == 0):
                    continue
                per = 1 if kind == SUM else rng.choice([1, 2, 4, 8])
                nt = 1 if kind == SUM else rng.randint(1, 40)
                seq.append((kind, nt, per, kind != SUM))
    return seq


def run(worklist_exe, seqs, order, ord_, cls, cap):
    lines = [f"{len(seqs)} {order} {cap}"]
    for s in seqs:
        lines.append(" ".join([str(len(s))] + [f"{nt} {per} {int(ch)}" for _, nt, per, ch in s]))
    lines.append(" ".join(map(str, ord_)))
    lines.append(" ".join(map(str, cls)))
    out = subprocess.run([worklist_exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True).stdout
    skew, slots, tickets, groups = None, [], None, []
    for ln in out.splitlines():
        f = ln.split()
        if f[0] == "skew":
            skew = [int(x) for x in f[1:]]
        elif f[0] == "slot":
            slots.append(tuple(int(x) for x in f[1:]))
        elif f[0] == "tickets":
            tickets = int(f[1])
        elif f[0] == "group":
            groups.append([int(x) for x in f[1:]])
    return skew, slots, tickets, groups


def simulate_queue(slots, seqs, ctas, rng):
    """Ticket queue with `ctas` CTAs acting in random order: a CTA takes the
    next ticket, and finishes it once its pass instance's dependency has all
    its tiles done.  Returns True if every ticket finishes, False on a state
    where no CTA can act (deadlock)."""
    tick_owner = []  # ticket -> (slot index, tiles in the ticket)
    for k, (mem, item, _, _, _) in enumerate(slots):
        _, nt, per, _ = seqs[mem][item]
        for t in range(math.ceil(nt / per)):
            tick_owner.append((k, min(per, nt - t * per)))
    done = [0] * len(slots)
    head = 0
    held = [None] * ctas
    finished = 0
    while finished < len(tick_owner):
        movable = []
        for c in range(ctas):
            if held[c] is None:
                if head < len(tick_owner):
                    movable.append(c)
            else:
                k, _ = tick_owner[held[c]]
                dep, need = slots[k][3], slots[k][4]
                if dep < 0 or done[dep] >= need:
                    movable.append(c)
        if not movable:
            return False
        c = rng.choice(movable)
        if held[c] is None:
            held[c] = head
            head += 1
        else:
            k, tiles = tick_owner[held[c]]
            done[k] += tiles
            held[c] = None
            finished += 1
    return True


@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_persistent_work_list(worklist_exe, order, seed):
    rng = random.Random(seed * 10 + order)
    m = rng.randint(1, 13)
    stages = rng.choice([2, 4])
    nsteps = rng.randint(1, 3)
    seqs = [member_sequence(rng, nsteps, stages) for _ in range(m)]
    ord_ = list(range(m))
    if order >= 1:
        rng.shuffle(ord_)  # any permutation (the library sorts by grid size)
    skew, slots, tickets, _ = run(worklist_exe, seqs, order, ord_, list(range(m)), 1)

    # skew: none, or the position in the member order modulo 6
    assert skew == ([0] * m if order < 2 else [ord_.index(i) % 6 for i in range(m)])
    # every pass instance exactly once, each member's in its own order
    assert sorted((s[0], s[1]) for s in slots) == [(i, k) for i in range(m) for k in range(len(seqs[i]))]
    for i in range(m):
        assert [s[1] for s in slots if s[0] == i] == list(range(len(seqs[i])))
    # level by level (level = item + skew), members in `ord` order within a level
    keys = [(s[1] + skew[s[0]], ord_.index(s[0])) for s in slots]
    assert keys == sorted(keys)
    # tickets: consecutive ranges, ceil(ntiles / per) each
    t = 0
    for mem, item, tick0, _, _ in slots:
        assert tick0 == t
        _, nt, per, _ = seqs[mem][item]
        t += math.ceil(nt / per)
    assert tickets == t
    # dependency: the member's previous chained pass instance, with its tile count
    for k, (mem, item, tick0, dep, need) in enumerate(slots):
        prev = [j for j in range(item) if seqs[mem][j][3]]
        if not prev:
            assert dep == -1 and need == 0
            continue
        assert slots[dep][0] == mem and slots[dep][1] == prev[-1]
        assert need == seqs[mem][prev[-1]][1]
        # the dependency's tickets all come before this pass instance's first
        d_mem, d_item, d_tick0 = slots[dep][:3]
        assert dep < k and d_tick0 + math.ceil(seqs[d_mem][d_item][1] / seqs[d_mem][d_item][2]) <= tick0
    # forward progress with any number of resident CTAs
    for ctas in (1, 2, 5, 64):
        assert simulate_queue(slots, seqs, ctas, random.Random(ctas))


def test_queue_simulation_detects_a_forward_dependency():
    # two passes of one member listed in the wrong order: the first waits for
    # the second, which no CTA can reach while one CTA holds the first ticket
    seqs = [[(ZINV, 2, 1, True), (YINV, 3, 1, True)]]
    slots = [(0, 1, 0, 1, 2), (0, 0, 3, -1, 0)]
    assert not simulate_queue(slots, seqs, 1, random.Random(0))


@pytest.mark.parametrize("cap", [1, 2, 4, 32])
def test_batched_groups(worklist_exe, cap):
    rng = random.Random(cap)
    m = 48
    cls = [rng.choice([0, 7, 9]) for _ in range(m)]
    _, _, _, groups = run(worklist_exe, [[] for _ in range(m)], 0, list(range(m)), cls, cap)
    assert sorted(j for g in groups for j in g) == list(range(m))
    placed = set()
    for g in groups:
        assert 1 <= len(g) <= cap and g == sorted(g)
        assert len({cls[j] for j in g}) == 1
        # a group starts at the first member not yet placed and takes the
        # next members of its class in order
        assert g[0] == min(set(range(m)) - placed)
        same = [j for j in range(m) if cls[j] == cls[g[0]] and j not in placed]
        assert g == same[:cap]
        placed.update(g)
