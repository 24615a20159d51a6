"""Hand-off protocol of the warp-specialized tensor-core kernel
(csrc/rom_tc_ws.cuh), checked on the CPU under random schedules.

The kernel's roles (8 tile warps, 4 helper warps, the asynchronous MMA and
copy engines) are modelled as coroutines that advance one step at a time in a
random order; MMAs of one warp complete in issue order but late, copies land
late.  mbarriers follow the parity rule of `mbarrier.try_wait.parity`: a wait
for parity p returns once the number of completed phases has the other
parity, so it is well defined only for the current phase and the one before
it.  Every data hazard the barriers guard is asserted:
  - a fold reads the accumulators of a chunk before its MMAs completed, or
    while MMAs of the next chunk run;
  - MMAs of the next chunk start before all four lane quarters were folded;
  - the residual reads w P or the tables before they were written / landed;
  - a w P buffer, a staging buffer or a B-operand image is overwritten while
    a reader may still use it; an A buffer is rewritten while MMAs read it;
  - nothing makes progress (a wait that never returns).
Two fold waits that are wrong pin the model's sensitivity: waiting for the
last k-step's commit on a per-buffer barrier (two phases per chunk) lets the
fold run early, and waiting for its two phases in turn blocks for good.

Timeouts: every wait of the kernels gives up after a bounded time.  The model
injects such timeouts at random blocked polls.  After the first one the CTA's
error flag is set: no wait blocks any more, no MMA or bulk copy is issued,
and the data hazards above are expected (the points are marked as timed out),
but every role must still finish, and TMEM may be freed only once every MMA
the tile warps issued has completed and every copy has landed (the drain at
the end of the kernels).  Leaving the drain out is caught.
The single-role kernel (csrc/rom_tc.cuh: 8 warps, a CTA barrier per chunk)
is modelled too; its earlier per-buffer fold wait passes early whenever a
warp is two k-steps behind, which random schedules reach.
"""
import random

import pytest

NW, NH, KSC = 8, 4, 4


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phases = count, count, 0

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.phases += 1
            self.pending = self.count

    def passed(self, parity):
        return (self.phases & 1) != parity


class NamedBarrier:
    def __init__(self, count):
        self.count, self.arrived, self.generation = count, 0, 0


class Hazard(AssertionError):
    pass


def run_schedule(seed, n_tiles, nch, fold_wait='chunk', max_steps=400_000, timeout_at=None, drain=True,
                 latency=30, clock=False, nw=NW, ksc=KSC, fk=None, defer=False, nh=NH, tile_fold=None):
    """timeout_at: the first wait still blocked at or after this model time
    runs out.  Returns True when a timeout was injected; raises Hazard.
    nw tile warps, ksc k-steps per chunk, a fold every fk k-steps (default:
    once per chunk, the warp-specialized kernel; the wide kernel folds every
    2 or 4 k-steps with 3 or 5 tile warps).  defer: a group's first k-step
    is issued together with its second, after both A buffers are built (the
    wide kernel).  nh helper warps.  tile_fold: one fold barrier per tile,
    arrived at as each tile is folded ('own': each tile warp waits on its
    tile's barrier, the wide kernel; 'first': every tile warp waits on tile
    0's barrier, a wrong wait); None: one fold barrier after all tiles (the
    warp-specialized kernel)."""
    fk = ksc if fk is None else fk
    ngr = ksc // fk
    rng = random.Random(seed)
    err = [False]                        # the CTA's timeout flag
    inflight = {'mma': [0] * nw, 'copy': 0}
    bx = [Barrier(1), Barrier(1)]
    commit = [[Barrier(1), Barrier(1)] for _ in range(nw)]
    chunk = [Barrier(1) for _ in range(nw)]
    staged = [Barrier(nh), Barrier(nh)]   # one arrival per helper warp's copies
    wp = [Barrier(nw), Barrier(nw)]
    res = [Barrier(nh), Barrier(nh)]
    fold = Barrier(nh)
    tfold = [Barrier(nh) for _ in range(nw)]
    named = {0: NamedBarrier(nw + nh), 1: NamedBarrier(nh), 2: NamedBarrier(nw)}
    events = []        # (time, action) of the asynchronous engines
    last_mma = {}      # per warp: completion time of its latest MMA group
    now = [0]
    mma_done, mma_issued, folded = set(), set(), {}   # per (warp, fold group)
    pending = set()                                    # (warp, k-step) built, MMAs not issued yet
    chunk_done = set()                                 # per (warp, chunk)
    wp_written, res_done, landed, readers, y_busy = {}, {}, set(), {}, {}

    def check(cond, what):
        # data hazards are expected once a wait timed out (the points are
        # marked, their outputs discarded)
        if not cond and not err[0]:
            raise Hazard(what)

    def later(action, warp=None):
        t = now[0] + rng.randint(1, latency)
        if warp is not None:                 # one warp's MMAs complete in order
            t = max(t, last_mma.get(warp, 0) + 1)
            last_mma[warp] = t
        events.append((t, action))

    def wait(bar, parity):
        while not bar.passed(parity) and not err[0]:
            if timeout_at is not None and now[0] >= timeout_at:   # the bounded wait runs out
                err[0] = True
                return
            yield

    def drain_wait(cond):
        # the end-of-kernel drain: bounded too, but the engines always finish
        while not cond():
            yield

    def sync(i):
        nb = named[i]
        gen = nb.generation
        nb.arrived += 1
        if nb.arrived == nb.count:
            nb.arrived, nb.generation = 0, gen + 1
        while nb.generation == gen:
            yield

    def stage(g):
        if err[0]:                           # nothing is issued after a timeout
            return
        b = g & 1
        check(readers.get(g - 2, 0) == 0, 'tables of chunk %d overwritten while read' % (g - 2))
        if g >= 2:
            check(all((w, g - 2) in chunk_done for w in range(nw)), 'B image of chunk %d overwritten' % (g - 2))

        def land():
            inflight['copy'] -= 1
            landed.add(g)
            for _ in range(nh):
                staged[b].arrive()

        def land_bx():
            inflight['copy'] -= 1
            bx[b].arrive()
        inflight['copy'] += 2
        later(land)
        later(land_bx)

    def group_wait(w, gr, sl):
        # the fold's wait for the MMAs of group gr (last k-step sl) of warp w
        if fold_wait == 'chunk':
            yield from wait(chunk[w], gr & 1)
        elif fold_wait == 'buffer':
            yield from wait(commit[w][sl & 1], (sl >> 1) & 1)
        else:  # both phases of the buffer barrier in turn
            yield from wait(commit[w][sl & 1], ((sl >> 1) & 1) ^ 1)
            yield from wait(commit[w][sl & 1], (sl >> 1) & 1)

    def helper(h):
        gc = gs = gg = 0
        for _ in range(n_tiles):
            if h == 0:
                stage(gc)
                if nch > 1:
                    stage(gc + 1)
            yield from sync(0)
            for ch in range(nch):
                g = gc + ch
                b = g & 1
                for gi in range(ngr):
                    gr = gg + ch * ngr + gi
                    sl = gs + ch * ksc + gi * fk + fk - 1       # the group's last k-step
                    if tile_fold:
                        for w in range(nw):
                            yield from group_wait(w, gr, sl)
                            check((w, gr) in mma_done, 'fold of group %d before its MMAs completed' % gr)
                            check((w, gr + 1) not in mma_issued, 'fold of group %d while group %d runs' % (gr, gr + 1))
                            folded.setdefault((w, gr), set()).add(h)
                            yield
                            tfold[w].arrive()
                        continue
                    for w in range(nw):
                        yield from group_wait(w, gr, sl)
                    for w in range(nw):
                        check((w, gr) in mma_done, 'fold of group %d before its MMAs completed' % gr)
                        check((w, gr + 1) not in mma_issued, 'fold of group %d while group %d runs' % (gr, gr + 1))
                        folded.setdefault((w, gr), set()).add(h)
                        yield
                    fold.arrive()
                yield from wait(wp[b], (g >> 1) & 1)
                yield from wait(staged[b], (g >> 1) & 1)
                check(len(wp_written.get(g, ())) == nw, 'residual of chunk %d before w P' % g)
                check(g in landed, 'residual of chunk %d before its tables' % g)
                readers[g] = readers.get(g, 0) + 1
                yield
                readers[g] -= 1
                res_done.setdefault(g, set()).add(h)
                res[b].arrive()
                if ch + 2 < nch:
                    yield from sync(1)
                    if h == 0:
                        stage(g + 2)
            yield from sync(0)
            gc += nch
            gs += nch * ksc
            gg += nch * ngr
            yield from sync(0)
        if drain and h == 0:
            yield from drain_wait(lambda: inflight['copy'] == 0)
        yield from sync(0)                   # the CTA barrier before TMEM is freed
        if h == 0:
            free_tmem()

    def free_tmem():
        if any(inflight['mma']) or inflight['copy']:
            raise Hazard('TMEM freed or CTA ended with MMAs or copies in flight')

    def tile(w):
        gc = gs = gg = 0
        for _ in range(n_tiles):
            yield from sync(2)
            yield from sync(0)
            for ch in range(nch):
                g = gc + ch
                b = g & 1
                yield from wait(staged[b], (g >> 1) & 1)
                if g >= 2:
                    yield from wait(res[b], ((g >> 1) & 1) ^ 1)
                check(g in landed, 'law of chunk %d before its tables' % g)
                check(g < 2 or len(res_done.get(g - 2, ())) == nh, 'w P of chunk %d overwritten' % (g - 2))
                readers[g] = readers.get(g, 0) + 1
                wp_written.setdefault(g, set()).add(w)
                wp[b].arrive()
                for ks in range(ksc):
                    s = gs + ch * ksc + ks
                    gr = gg + ch * ngr + ks // fk
                    yb = s & 1
                    if s >= 2:
                        yield from wait(commit[w][yb], ((s - 2) >> 1) & 1)
                    check(y_busy.get((w, yb), 0) == 0, 'A buffer rewritten while MMAs read it')
                    check((w, s) not in pending, 'A buffer rewritten before its MMAs were issued')
                    pending.add((w, s))
                    yield
                    kg = ks % fk
                    if defer and kg == 0:
                        continue                     # issued with the next k-step
                    first = (kg == 1) if defer else (kg == 0)
                    if ks == (1 if defer else 0):
                        yield from wait(bx[b], (g >> 1) & 1)
                    if first and gr >= 1:
                        fb = fold if not tile_fold else tfold[w if tile_fold == 'own' else 0]
                        yield from wait(fb, (gr - 1) & 1)
                        check(len(folded.get((w, gr - 1), ())) == nh, 'MMAs of group %d before the fold' % gr)
                    if err[0]:                   # no MMA is issued after a timeout
                        pending.discard((w, s))
                        pending.discard((w, s - 1))
                        continue
                    for si in ((s - 1, s) if (defer and kg == 1) else (s,)):
                        pending.discard((w, si))
                        ybi = si & 1
                        mma_issued.add((w, gr))
                        y_busy[(w, ybi)] = y_busy.get((w, ybi), 0) + 1
                        glast = si == s and kg == fk - 1
                        clast = si == s and ks == ksc - 1
                        inflight['mma'][w] += 1

                        def complete(w=w, yb=ybi, g=g, gr=gr, glast=glast, clast=clast):
                            inflight['mma'][w] -= 1
                            y_busy[(w, yb)] -= 1
                            commit[w][yb].arrive()
                            if glast:
                                mma_done.add((w, gr))
                                chunk[w].arrive()
                            if clast:
                                chunk_done.add((w, g))
                        later(complete, warp=w)
                readers[g] -= 1
            yield from sync(0)
            gc += nch
            gs += nch * ksc
            gg += nch * ngr
            yield from sync(0)
        if drain:                            # commit + wait: all of this warp's MMAs completed
            yield from drain_wait(lambda: inflight['mma'][w] == 0)
        yield from sync(0)

    agents = [helper(h) for h in range(nh)] + [tile(w) for w in range(nw)]
    alive = list(range(len(agents)))
    steps = 0
    while alive:
        steps += 1
        check(steps < max_steps, 'no progress')
        now[0] += 1
        due = [e for e in events if e[0] <= now[0]]
        for e in due:
            events.remove(e)
            e[1]()
        i = rng.choice(alive)
        try:
            next(agents[i])
        except StopIteration:
            alive.remove(i)
    return now[0] if clock else err[0]


@pytest.mark.parametrize('seed', range(40))
def test_protocol_is_hazard_free(seed):
    # a CTA's contiguous share of the points may hold no tile at all (fewer
    # points than CTAs): n_tiles = 0 only drains
    assert not run_schedule(seed, n_tiles=seed % 4, nch=1 + (seed // 3) % 6)


@pytest.mark.parametrize('seed', range(40))
@pytest.mark.parametrize('nw,ksc,fk,nh', [(3, 8, 2, 8), (3, 8, 2, 4), (5, 4, 2, 4), (5, 4, 4, 4)])
def test_wide_kernel_protocol_is_hazard_free(seed, nw, ksc, fk, nh):
    # the wide kernel: fewer tile warps, fold groups of fk k-steps within a
    # chunk (chunk and fold barriers advance once per group), a fold barrier
    # per tile, 4 or 8 helper warps
    assert not run_schedule(seed, n_tiles=seed % 4, nch=1 + (seed // 3) % 5, nw=nw, ksc=ksc, fk=fk, defer=True,
                            nh=nh, tile_fold='own')


@pytest.mark.parametrize('seed', range(20))
def test_wide_kernel_timeouts_end_after_a_drain(seed):
    nt, nch = 1 + seed % 3, 1 + (seed // 3) % 5
    latency = 30 if seed % 2 else 400
    kw = dict(nw=3, ksc=8, fk=2, defer=True, nh=8, tile_fold='own')
    span = run_schedule(seed, nt, nch, latency=latency, clock=True, **kw)
    r = random.Random(seed)
    at = r.randrange(span) if seed % 3 else max(0, span - r.randrange(1, latency))
    run_schedule(seed, nt, nch, latency=latency, timeout_at=at, **kw)


def test_wide_kernel_wrong_fold_wait_is_caught():
    # with fold groups of 4 k-steps, waiting on the per-buffer commit barrier
    # of the group's last k-step instead of the group barrier lets a fold run
    # early (with groups of 2 k-steps each buffer barrier advances once per
    # group, and that wait would be as good as the group barrier)
    hits = 0
    for seed in range(6):
        try:
            run_schedule(seed, n_tiles=2, nch=3, fold_wait='buffer', max_steps=60_000, nw=5, ksc=4, fk=4, defer=True,
                         tile_fold='own')
        except Hazard as e:
            assert 'before its MMAs completed' in str(e)
            hits += 1
    assert hits > 0


@pytest.mark.parametrize('seed', range(30))
def test_timeouts_end_the_kernel_after_a_drain(seed):
    # random timeouts: every role finishes, and nothing is in flight when
    # TMEM is freed
    # (the timeout time is uniform over the run, or within the last MMA
    # latency of its end, where MMAs of the last chunk are still in flight)
    nt, nch = 1 + seed % 3, 1 + (seed // 3) % 6
    latency = 30 if seed % 2 else 400
    span = run_schedule(seed, nt, nch, latency=latency, clock=True)
    r = random.Random(seed)
    at = r.randrange(span) if seed % 3 else max(0, span - r.randrange(1, latency))
    run_schedule(seed, nt, nch, latency=latency, timeout_at=at)


def test_missing_drain_is_caught():
    # timeouts during the last chunks, without the drain: some schedules free
    # TMEM while MMAs still run
    hits = 0
    for seed in range(6):
        span = run_schedule(seed, n_tiles=2, nch=4, latency=400, clock=True)
        for back in range(100, 1600, 100):
            try:
                run_schedule(seed, n_tiles=2, nch=4, latency=400, drain=False, timeout_at=span - back)
            except Hazard as e:
                assert 'in flight' in str(e)
                hits += 1
    assert hits > 0


@pytest.mark.parametrize('variant, what', [('buffer', 'before its MMAs completed'), ('two-phase', 'no progress')])
def test_wrong_fold_waits_are_caught(variant, what):
    hits = 0
    for seed in range(6):
        try:
            run_schedule(seed, n_tiles=2, nch=4, fold_wait=variant, max_steps=60_000)
        except Hazard as e:
            assert what in str(e)
            hits += 1
    assert hits > 0


def run_single_role(seed, n_tiles, nch, fold_wait='chunk', max_steps=400_000, timeout_at=None, drain=True,
                    latency=30, clock=False):
    """Protocol of the single-role kernel (csrc/rom_tc.cuh): 8 warps, each
    issuing its own tile's MMAs per k-step and folding one lane quarter of
    every tile after the chunk, then a CTA barrier; returns nothing, raises
    Hazard."""
    rng = random.Random(seed)
    commit = [[Barrier(1), Barrier(1)] for _ in range(NW)]
    chunk = [Barrier(1) for _ in range(NW)]
    cta = NamedBarrier(NW)
    events, last_mma, now = [], {}, [0]
    mma_done, folds = set(), {}
    err, inflight = [False], [0] * NW

    def check(cond, what):
        if not cond and not err[0]:
            raise Hazard(what)

    def later(action, warp):
        t = max(now[0] + rng.randint(1, latency), last_mma.get(warp, 0) + 1)
        last_mma[warp] = t
        events.append((t, action))

    def wait(bar, parity):
        while not bar.passed(parity) and not err[0]:
            if timeout_at is not None and now[0] >= timeout_at:
                err[0] = True
                return
            yield

    def sync():
        gen = cta.generation
        cta.arrived += 1
        if cta.arrived == cta.count:
            cta.arrived, cta.generation = 0, gen + 1
        while cta.generation == gen:
            yield

    def warp(w):
        gstep = gchunk = 0
        for _ in range(n_tiles):
            for ch in range(nch):
                for ks in range(KSC):
                    s = gstep + ks
                    if s >= 2:
                        yield from wait(commit[w][s & 1], ((s - 2) >> 1) & 1)
                    yield
                    check(all(folds.get((t, gchunk - 1), 0) == NW for t in range(NW)) or ch == 0 and gchunk == 0,
                          'MMAs before the fold of the previous chunk')
                    if err[0]:                   # no MMA is issued after a timeout
                        continue
                    last = ks == KSC - 1
                    inflight[w] += 1

                    def complete(w=w, s=s, g=gchunk, last=last):
                        inflight[w] -= 1
                        commit[w][s & 1].arrive()
                        if last:
                            mma_done.add((w, g))
                            chunk[w].arrive()
                    later(complete, w)
                gstep += KSC
                sl = gstep - 1
                for w2 in range(NW):
                    if fold_wait == 'chunk':
                        yield from wait(chunk[w2], gchunk & 1)
                    else:
                        yield from wait(commit[w2][sl & 1], (sl >> 1) & 1)
                for t in range(NW):
                    check((t, gchunk) in mma_done, 'fold of chunk %d before its MMAs completed' % gchunk)
                    folds[(t, gchunk)] = folds.get((t, gchunk), 0) + 1
                    yield
                yield from sync()
                gchunk += 1
        if drain:                                # commit + bounded wait
            while inflight[w]:
                yield
        yield from sync()
        if w == 0 and any(inflight):
            raise Hazard('TMEM freed with MMAs in flight')

    agents = [warp(w) for w in range(NW)]
    alive = list(range(NW))
    steps = 0
    while alive:
        steps += 1
        check(steps < max_steps, 'no progress')
        now[0] += 1
        due = [e for e in events if e[0] <= now[0]]
        for e in due:
            events.remove(e)
            e[1]()
        i = rng.choice(alive)
        try:
            next(agents[i])
        except StopIteration:
            alive.remove(i)
    return now[0] if clock else err[0]


@pytest.mark.parametrize('seed', range(20))
def test_single_role_protocol_is_hazard_free(seed):
    run_single_role(seed, n_tiles=seed % 3, nch=1 + seed % 5)


@pytest.mark.parametrize('seed', range(20))
def test_single_role_timeouts_end_after_a_drain(seed):
    nt, nch = 1 + seed % 2, 1 + seed % 5
    span = run_single_role(seed, nt, nch, latency=400, clock=True)
    for back in range(50, span, max(50, span // 10)):
        run_single_role(seed, nt, nch, latency=400, timeout_at=span - back)


def test_single_role_missing_drain_is_caught():
    hits = 0
    for seed in range(6):
        span = run_single_role(seed, 1, 4, latency=400, clock=True)
        for back in range(50, 1500, 50):
            try:
                run_single_role(seed, 1, 4, latency=400, drain=False, timeout_at=span - back)
            except Hazard as e:
                assert 'in flight' in str(e)
                hits += 1
    assert hits > 0


def test_single_role_buffer_wait_is_caught():
    # waiting for the last k-step's commit on its per-buffer barrier passes
    # early whenever another warp is two k-steps behind
    hits = 0
    for seed in range(30):
        try:
            run_single_role(seed, n_tiles=1, nch=4, fold_wait='buffer')
        except Hazard as e:
            assert 'before its MMAs completed' in str(e)
            hits += 1
    assert hits > 0


def test_wide_kernel_wrong_tile_fold_wait_is_caught():
    # every tile warp waiting on tile 0's fold barrier instead of its own
    # issues MMAs onto accumulators the helpers have not folded yet
    hits = 0
    for seed in range(8):
        try:
            run_schedule(seed, n_tiles=2, nch=3, max_steps=60_000, nw=3, ksc=8, fk=2, defer=True, nh=8,
                         tile_fold='first')
        except Hazard as e:
            assert 'before the fold' in str(e) or 'while group' in str(e)
            hits += 1
    assert hits > 0
