"""Discrete-event model of the carry kernel's mbarrier protocol (the
block-parallel tensor-core form): four power-panel slots, two OUTPUT-operand
(W) slots, two carry groups, separate STATE and OUTPUT issuers, a panel
copier, and an epilogue role that drains each (template, batch) in order.
A carry group either releases its STATE columns after its last read, while
it makes W (one stream), or reads every chunk's sum first and releases them
before it waits for its W slot (two streams); both orders are checked. The
roles and their waits restate the kernel's; MMAs and copies complete at
issue (once issued they wait on nothing), so every interleaving the random
scheduler picks is a possible execution order. The model checks: no
deadlock, no phase aliasing (a wait never sees its barrier two phases
ahead), the strain-buffer refill margin (panel j ready implies OUTPUT j - 4
finished), and that each tile's batches are carried in order."""
import random


KP, KW = 4, 2


class Bar:
    def __init__(s, name, count):
        s.name, s.count, s.pending, s.C = name, count, count, 0

    def arrive(s, n=1):
        s.pending -= n
        assert s.pending >= 0, s.name
        if s.pending == 0:
            s.C += 1
            s.pending = s.count


def jobs(n_carry, grid, bid, tile_ptr, n_batches):
    j = e = 0
    multi = n_batches > 1
    out = []
    for ti in range(bid, n_carry, grid):
        t0, t1 = tile_ptr[ti], tile_ptr[ti + 1]
        for b0 in range(n_batches):
            for tile in range(t0, t1):
                g = ((tile - t0) & 1) if multi else (j & 1)
                out.append(dict(t=ti, b0=b0, tile=tile, first=tile == t0, last=tile == t1 - 1, j=j, e=e,
                                s=j % KP, w=j % KW, g=g))
                j += 1
            e += 1
    return out


def run(JOBS, seed, u_first=False, drop=None):
    """drop: a wait left out ('sfree' STATE issuer, 'ofree' OUTPUT issuer,
    'wfull' OUTPUT issuer, 'pfree' copier, 'ofull' epilogue, 'wfree' and
    'sfull' carry), to show that the model catches it."""
    B = {}

    def bar(n, c):
        B[n] = Bar(n, c)
    for i in range(KP):
        bar(f'pfull{i}', 1); bar(f'pfree{i}', 1)
    for i in range(KW):
        bar(f'wfull{i}', 128); bar(f'wfree{i}', 1)
    for i in range(2):
        bar(f'sfull{i}', 1); bar(f'sfree{i}', 128); bar(f'ofull{i}', 1); bar(f'ofree{i}', 128)
    vlog = {}
    out_done = set()

    def ready(name, idx):
        """Has phase idx of the barrier completed? (parity test, with an
        aliasing check: the barrier may not be two phases ahead)."""
        b = B[name]
        assert b.C <= idx + 1, ('alias', name, b.C, idx)
        return b.C >= idx + 1

    def W(name, idx):
        return ('wait', name, idx)

    def state_issuer():
        n_sf = [0, 0]; used = [False, False]
        for J in JOBS:
            g, s = J['g'], J['s']
            if used[g]:
                if drop != 'sfree':
                    yield W(f'sfree{g}', n_sf[g])
                n_sf[g] += 1
            used[g] = True
            yield W(f'pfull{s}', J['j'] // KP)
            # panel J ready => OUTPUT(J - KP) complete (its slot was freed)
            assert J['j'] < KP or (J['j'] - KP) in out_done, ('refill margin', J['j'])
            B[f'sfull{g}'].arrive()

    def output_issuer():
        n_of = [0, 0]
        for J in JOBS:
            ob, w, s = J['e'] & 1, J['w'], J['s']
            if J['first'] and J['e'] >= 2:
                if drop != 'ofree':
                    yield W(f'ofree{ob}', n_of[ob])
                n_of[ob] += 1
            if drop != 'wfull':
                yield W(f'wfull{w}', J['j'] // KW)
            B[f'wfree{w}'].arrive(); B[f'pfree{s}'].arrive()
            if J['last']:
                B[f'ofull{ob}'].arrive()
            out_done.add(J['j'])

    def copier():
        for J in JOBS:
            s = J['s']
            use = J['j'] // KP
            if use > 0 and drop != 'pfree':
                yield W(f'pfree{s}', use - 1)
            B[f'pfull{s}'].arrive()

    def epilogue():
        for J in JOBS:
            if not J['last']:
                continue
            ob = J['e'] & 1
            if drop != 'ofull':
                yield W(f'ofull{ob}', J['e'] >> 1)
            B[f'ofree{ob}'].arrive(128)

    def carry(grp):
        n_state = 0
        for J in JOBS:
            if J['g'] != grp:
                continue
            w = J['w']
            if drop != 'sfull':
                yield W(f'sfull{grp}', n_state)
            n_state += 1
            use = J['j'] // KW
            if u_first:
                B[f'sfree{grp}'].arrive(128)
            if use > 0 and drop != 'wfree':
                yield W(f'wfree{w}', use - 1)
            if not u_first:
                B[f'sfree{grp}'].arrive(128)
            vlog.setdefault((J['t'], J['tile']), []).append(J['b0'])
            B[f'wfull{w}'].arrive(128)

    roles = [state_issuer(), output_issuer(), copier(), epilogue(), carry(0), carry(1)]
    n = len(roles)
    st = [None] * n; done = [False] * n
    rng = random.Random(seed)

    def step(i):
        try:
            st[i] = next(roles[i])
        except StopIteration:
            done[i] = True
    for i in range(n):
        step(i)
    while not all(done):
        go, polls = [], []
        for i in range(n):
            if done[i]:
                continue
            if st[i][0] == 'poll':
                polls.append(i)
            elif ready(st[i][1], st[i][2]):
                go.append(i)
        if not go and not polls:
            raise AssertionError('deadlock ' + str(st))
        i = rng.choice(go + polls)
        if i in polls:
            snap = [(k, v.C, v.pending) for k, v in B.items()]
            step(i)
            if not go and not done[i] and [(k, v.C, v.pending) for k, v in B.items()] == snap \
                    and st[i][0] == 'poll':
                # only pollers left and the poll changed nothing: check that
                # no waiter can ever be released
                raise AssertionError('deadlock (poll) ' + str(st))
        else:
            step(i)
    for k, v in vlog.items():
        assert v == sorted(v), (k, v)
    assert len(out_done) == len(JOBS)


def test_carry_protocol_all_job_shapes():
    """Templates of 1-6 tiles, 1-7 templates per CTA, 1-3 CTAs, 1-8 batches
    per push, several random interleavings each."""
    cnt = 0
    for pat in [[1], [2], [3], [4], [5], [1, 2], [3, 1, 2], [5, 1, 1, 4], [2, 3], [1, 1, 1, 6]]:
        for n_carry in [1, 2, 3, 5, 7]:
            for grid in [1, 2, 3]:
                for nb in [1, 2, 3, 4, 5, 8]:
                    tp = [0]
                    for i in range(n_carry):
                        tp.append(tp[-1] + pat[i % len(pat)])
                    for bid in range(min(grid, n_carry)):
                        J = jobs(n_carry, grid, bid, tp, nb)
                        for seed in range(6):
                            run(J, seed, u_first=bool(seed & 1))
                            cnt += 1
    assert cnt > 9000


def test_carry_protocol_catches_each_missing_wait():
    """The model is not vacuous: leaving out any one wait of any role breaks
    one of its checks for some job shape and interleaving."""
    shapes = []
    for pat in [[1], [2], [3], [1, 2], [5, 1, 1, 4]]:
        for n_carry in [3, 7]:
            for nb in [1, 2, 5]:
                tp = [0]
                for i in range(n_carry):
                    tp.append(tp[-1] + pat[i % len(pat)])
                shapes.append(jobs(n_carry, 1, 0, tp, nb))
    for drop in ['sfree', 'ofree', 'wfull', 'pfree', 'ofull', 'sfull', 'wfree']:
        for u_first in (False, True):
            caught = False
            for J in shapes:
                for seed in range(8):
                    try:
                        run(J, seed, u_first=u_first, drop=drop)
                    except AssertionError:
                        caught = True
                        break
                if caught:
                    break
            assert caught, (drop, u_first)
