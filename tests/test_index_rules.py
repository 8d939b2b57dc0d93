"""Host-side checks of the index and coefficient rules the kernels use (the
GPU parity tests check that the kernels follow them):

* the x-compacted neighbour indices of a parity site (Sec. 3.3-3.4), written as
  the hopping kernels compute them, against lex/2 of x +- mu computed from the
  coordinates, for extents down to 2;
* the fused kernel's wavefront task order: each first-hop task A(t) and
  second-hop task B(t) appears once, and every B(t) comes after A(t-1), A(t),
  A(t+1), for every t extent and lookahead (this is what makes its bounded
  waits deadlock-free);
* the float-float kernel's run-time projector table: unit factors c0, c1 and
  spin indices j0, j1 with h = psi_up + c psi_j, and d2, d3, k2, k3 with
  out_dn += d chi_k, against (1 - S gamma_mu) in the chiral basis of Eq. 1.
"""

import itertools

import numpy as np
import pytest


def kernel_neighbours(dims, out_parity, i):
    """The compact neighbour indices as the hopping kernels compute them."""
    lx, ly, lz, lt = dims
    lxh = lx // 2
    xh, rem = i % lxh, i // lxh
    y, rem = rem % ly, rem // ly
    z, t = rem % lz, rem // lz
    par = (y + z + t + out_parity) & 1
    sy, sz, st = lxh, lxh * ly, lxh * ly * lz
    row = i - xh
    xp = (0 if xh + 1 == lxh else xh + 1) if par else xh
    xm = xh if par else (lxh - 1 if xh == 0 else xh - 1)
    return {
        (0, 1): row + xp, (0, -1): row + xm,
        (1, 1): i + (-(ly - 1) * sy if y + 1 == ly else sy), (1, -1): i + ((ly - 1) * sy if y == 0 else -sy),
        (2, 1): i + (-(lz - 1) * sz if z + 1 == lz else sz), (2, -1): i + ((lz - 1) * sz if z == 0 else -sz),
        (3, 1): i + (-(lt - 1) * st if t + 1 == lt else st), (3, -1): i + ((lt - 1) * st if t == 0 else -st),
    }, (2 * xh + par, y, z, t)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 6, 2), (4, 2, 2, 8), (6, 4, 4, 2), (8, 6, 2, 4)])
@pytest.mark.parametrize("out_parity", [0, 1])
def test_compact_neighbour_indices(dims, out_parity):
    lx, ly, lz, lt = dims
    vh = lx * ly * lz * lt // 2
    for i in range(vh):
        nb, (x, y, z, t) = kernel_neighbours(dims, out_parity, i)
        assert (x + y + z + t) % 2 == out_parity
        assert ((t * lz + z) * ly + y) * lx + x == 2 * i + (x % 2)  # lex/2 == i
        c = [x, y, z, t]
        for (mu, sgn), n in nb.items():
            d = list(c)
            d[mu] = (d[mu] + sgn) % dims[mu]
            lex = ((d[3] * lz + d[2]) * ly + d[1]) * lx + d[0]
            assert n == lex // 2, (dims, out_parity, i, mu, sgn)


def fused_task(L, D, k):
    """Slice task k of the fused kernel's queue: ('A'|'B', t)."""
    if k == 0:
        return ("A", L - 1)
    if k <= D:
        return ("A", k - 1)
    kp, pairs = k - (D + 1), L - 1 - D
    if kp < 2 * pairs:
        return ("B", kp >> 1) if kp & 1 else ("A", (kp >> 1) + D)
    return ("B", pairs + (kp - 2 * pairs))


def test_fused_queue_order():
    for L in range(2, 131, 2):
        for D0 in range(1, 70):
            D = max(1, min(D0, L - 1))  # as the host clamps it
            seq = [fused_task(L, D, k) for k in range(2 * L)]
            assert sorted(seq) == sorted([("A", t) for t in range(L)] + [("B", t) for t in range(L)])
            pos = {x: n for n, x in enumerate(seq)}
            for t in range(L):
                for u in ((t - 1) % L, t, (t + 1) % L):
                    assert pos[("A", u)] < pos[("B", t)], (L, D, t, u)


def dir_coef(mu, S):
    """The float-float kernel's table: (c0, j0, c1, j1, d2, k2, d3, k3), unit
    factors as complex numbers."""
    sp = S > 0

    def unit(rot, neg):
        return (1j if rot else 1) * (-1 if neg else 1)

    rows = {
        0: (True, not sp, True, not sp, 3, 2, True, sp, True, sp, 1, 0),
        1: (False, not sp, False, sp, 3, 2, False, sp, False, not sp, 1, 0),
        2: (True, not sp, True, sp, 2, 3, True, sp, True, not sp, 0, 1),
        3: (False, sp, False, sp, 2, 3, False, sp, False, sp, 0, 1),
    }
    r0, n0, r1, n1, j0, j1, r2, n2, r3, n3, k2, k3 = rows[mu]
    return unit(r0, n0), j0, unit(r1, n1), j1, unit(r2, n2), k2, unit(r3, n3), k3


@pytest.mark.parametrize("mu,S", list(itertools.product(range(4), (1, -1))))
def test_float_float_projector_table(oracle_lib, mu, S):
    """(1 - S gamma_mu) psi has upper components h = psi_up + c psi_j and lower
    components -S A^dag h; the kernel adds d_2 chi_{k2}, d_3 chi_{k3} to the
    lower components of out for chi = U h, which must equal that lower part."""
    g = oracle_lib.gamma(mu)
    P = np.eye(4) - S * g
    rng = np.random.default_rng(10 * mu + (S > 0))
    psi = rng.normal(size=4) + 1j * rng.normal(size=4)
    full = P @ psi
    c0, j0, c1, j1, d2, k2, d3, k3 = dir_coef(mu, S)
    h = np.array([psi[0] + c0 * psi[j0], psi[1] + c1 * psi[j1]])
    assert np.allclose(full[:2], h)
    # the lower half of (1 - S gamma) psi, rebuilt from h as the kernel does
    assert np.allclose(full[2], d2 * h[k2]) and np.allclose(full[3], d3 * h[k3])


# ---------------------------------------------------------------- staged hop --
# The TMA-staged hopping kernel (csrc/hop_staged.cu) reads every operand of a
# tile of R rows from blocks it loaded into shared memory: seven spinor boxes
# and the tile's link block (packed once per gauge field: direction d = 2 mu + b
# of site s holds U_mu(x), or U_mu(x - mu) for b = 1). This model follows the
# kernel's tile, box and in-tile index arithmetic and checks that every value
# it reads is the neighbour spinor / link the hopping sum needs.

def staged_rows(lxh, ly, want=0):
    if lxh % 2:
        return 0
    ok = lambda r: r >= 2 and ly % r == 0 and r * lxh <= 64  # noqa: E731
    if want:
        return want if ok(want) else 0
    for r in range(64 // lxh, 1, -1):
        if ok(r):
            return r
    return 0


def staged_boxes(dims, rows, j):
    """Spinor boxes of tile j: region -> (first compact site, sites)."""
    lx, ly, lz, lt = dims
    lxh = lx // 2
    row0 = j * rows
    plane, y0 = divmod(row0, ly)
    t, z = divmod(plane, lz)

    def rs(z_, t_, y_):
        return ((t_ * lz + z_) * ly + y_) * lxh

    T, i0 = rows * lxh, row0 * lxh
    b = {"sp0": (i0, T), "sp1": (rs(z, t, (y0 - 1) % ly), lxh), "sp2": (rs(z, t, (y0 + rows) % ly), lxh),
         "sp3": (rs((z + 1) % lz, t, y0), T), "sp4": (rs((z - 1) % lz, t, y0), T),
         "sp5": (rs(z, (t + 1) % lt, y0), T), "sp6": (rs(z, (t - 1) % lt, y0), T)}
    return b, (y0, z, t, i0)


def staged_reads(dims, rows, geo, s, out_parity):
    """(direction, spinor region, index, link direction) as the consumers read them."""
    lxh = dims[0] // 2
    y0, z, t, _ = geo
    r, xh = divmod(s, lxh)
    par = (y0 + r + z + t + out_parity) & 1
    xp = (0 if xh + 1 == lxh else xh + 1) if par else xh
    xm = xh if par else (lxh - 1 if xh == 0 else xh - 1)
    rb = r * lxh
    out = [((0, 1), "sp0", rb + xp, 0), ((0, -1), "sp0", rb + xm, 1)]
    out.append(((1, 1), "sp0", rb + lxh + xh, 2) if r + 1 < rows else ((1, 1), "sp2", xh, 2))
    out.append(((1, -1), "sp0", rb - lxh + xh, 3) if r > 0 else ((1, -1), "sp1", xh, 3))
    out += [((2, 1), "sp3", s, 4), ((2, -1), "sp4", s, 5), ((3, 1), "sp5", s, 6), ((3, -1), "sp6", s, 7)]
    return out


def pack_link_blocks(dims, T, out_parity):
    """(field, compact index) stored at (tile, direction, site), as the packing
    kernel writes the link blocks."""
    lx, ly, lz, lt = dims
    lxh, vh = lx // 2, lx * ly * lz * lt // 2
    blk = {}
    for i in range(vh):
        xh, rem = i % lxh, i // lxh
        y, rem = rem % ly, rem // ly
        z, t = rem % lz, rem // lz
        par = (y + z + t + out_parity) & 1
        sy, sz, st = lxh, lxh * ly, lxh * ly * lz
        nb = [i - xh + (xh if par else (lxh - 1 if xh == 0 else xh - 1)),
              i + ((ly - 1) * sy if y == 0 else -sy), i + ((lz - 1) * sz if z == 0 else -sz),
              i + ((lt - 1) * st if t == 0 else -st)]
        for mu in range(4):
            blk[(i // T, 2 * mu, i % T)] = (2 * mu + out_parity, i)
            blk[(i // T, 2 * mu + 1, i % T)] = (2 * mu + (out_parity ^ 1), nb[mu])
    return blk


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 6), (8, 8, 8, 8), (16, 2, 4, 4),
                                  (12, 6, 4, 8), (4, 6, 2, 22), (32, 8, 2, 4), (24, 8, 2, 2),
                                  (48, 4, 2, 2)])
@pytest.mark.parametrize("out_parity", [0, 1])
@pytest.mark.parametrize("reverse", [False, True])
@pytest.mark.parametrize("want_rows", [0, 2])
def test_staged_tile_reads(dims, out_parity, reverse, want_rows):
    lx, ly, lz, lt = dims
    lxh, vh = lx // 2, lx * ly * lz * lt // 2
    rows = staged_rows(lxh, ly, want_rows)
    assert rows >= 2 and ly % rows == 0
    T = rows * lxh
    assert T <= 64 and vh % T == 0 and T % 2 == 0
    ntiles = vh // T
    blocks = pack_link_blocks(dims, T, out_parity)
    seen = np.zeros(vh, dtype=int)
    for jj in range(ntiles):
        j = ntiles - 1 - jj if reverse else jj
        boxes, geo = staged_boxes(dims, rows, j)
        jt = geo[3] // T  # the link block the producer copies
        for start, n in boxes.values():
            # every box lies inside the array (TMA would zero-fill, not wrap) and
            # its x coordinate (floats) is a multiple of 16 bytes
            assert 0 <= start and start + n <= vh
            assert (2 * start * 4) % 16 == 0 and 2 * n <= 256
        for s in range(T):
            i = geo[3] + s
            seen[i] += 1
            nb, _ = kernel_neighbours(dims, out_parity, i)
            for d, sreg, si, ld in staged_reads(dims, rows, geo, s, out_parity):
                start, n = boxes[sreg]
                assert 0 <= si < n
                assert start + si == nb[d], (dims, j, s, d)
                mu, sgn = d
                want = (2 * mu + out_parity, i) if sgn > 0 else (2 * mu + (out_parity ^ 1), nb[d])
                assert blocks[(jt, ld, s)] == want, (dims, j, s, d)
    assert (seen == 1).all()


def test_staged_layout_and_byte_count():
    """Stage regions are 128-byte aligned and disjoint, the ring fits in
    227 KB for the workload shapes, the link block's direction planes start on
    16-byte boundaries, and the mbarrier's expected byte count equals the bytes
    copied, for every tile shape the row rule allows."""
    for lxh, ly, want in itertools.product(range(2, 33, 2), range(2, 130, 2), (0, 2, 4)):
        rows = staged_rows(lxh, ly, want)
        if rows < 2:
            continue
        T = rows * lxh
        sizes = [96 * T, 96 * lxh, 96 * lxh] + [96 * T] * 4 + [576 * T, 96 * T]
        off, regions = 0, []
        for b in sizes:
            regions.append((off, off + b))
            off += (b + 127) // 128 * 128
        assert all(a % 128 == 0 for a, _ in regions)
        assert all(regions[k][1] <= regions[k + 1][0] for k in range(len(regions) - 1))
        assert all((72 * T * d) % 16 == 0 and (72 * T * d + 64 * T) % 16 == 0 for d in range(8))
        ring = {d: d * off + (2 * d + 6) * 8 for d in (2, 3, 4, 5)}
        if (lxh, ly) in ((16, 32), (24, 48), (12, 24), (8, 16), (4, 8)) and want == 0:
            assert ring[3] <= 227 * 1024, (lxh, ly)
        if (lxh, ly, want) == (16, 32, 2):
            assert ring[5] <= 227 * 1024
        assert sum(sizes) == 5 * 96 * T + 2 * 96 * lxh + 576 * T + 96 * T


# ------------------------------------------------- staged barrier protocol --
# mbarrier.try_wait.parity(P) succeeds when the phase of parity P has completed,
# i.e. when P differs from the parity of the phase in progress. A waiter that
# means phase n is therefore only right if the barrier is in phase n or n + 1
# when it tests. This simulates the multi-RHS staged kernel's producer, its
# link slots, its spinor ring and its consumer warps under random schedules
# and checks that condition at every test, and that every schedule finishes.

class _Barrier:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count


def _simulate_mrhs(ntiles, nrhs, ns, tpt, seed, land_p=0.3):
    rnd = np.random.default_rng(seed)
    full = [_Barrier(1) for _ in range(ns)]
    empty = [_Barrier(tpt) for _ in range(ns)]
    lfull = [_Barrier(1) for _ in range(2)]
    lempty = [_Barrier(tpt * nrhs) for _ in range(2)]
    ready = [_Barrier(1) for _ in range(ns * tpt)]
    nitems = ntiles * nrhs
    in_flight = []  # loads whose bytes have not landed: barriers to arrive on

    def test(bar, n):
        assert bar.phase in (n, n + 1), (bar.phase, n)
        return (n & 1) != (bar.phase & 1)

    def producer():
        for k in range(nitems):
            m, r = divmod(k, nrhs)
            if r == 0:
                if m >= 2:
                    while not test(lempty[m & 1], (m >> 1) - 1):
                        yield
                in_flight.append(lfull[m & 1])
            st, u = k % ns, k // ns
            if u >= 1:
                while not test(empty[st], u - 1):
                    yield
            in_flight.append(full[st])
            yield

    def consumer(team, q):
        g = team // tpt
        for k in range(g, nitems, ns):
            m, u = k // nrhs, k // ns
            while not test(lfull[m & 1], m >> 1):
                yield
            while not test(full[g], u):
                yield
            yield  # compute
            if q == 1:
                ready[team].arrive()
            else:
                while not test(ready[team], u):
                    yield
                empty[g].arrive()
                lempty[m & 1].arrive()
            yield

    actors = [producer()] + [consumer(t, q) for t in range(ns * tpt) for q in (0, 1)]
    live = list(range(len(actors)))
    steps = 0
    while live or in_flight:
        steps += 1
        assert steps < 200000, "no progress"
        if in_flight and (not live or rnd.random() < land_p):
            in_flight.pop(int(rnd.integers(len(in_flight)))).arrive()
            continue
        if not live:
            continue
        a = live[int(rnd.integers(len(live)))]
        try:
            next(actors[a])
        except StopIteration:
            live.remove(a)
    return steps


@pytest.mark.parametrize("ntiles,nrhs,ns,tpt", [(5, 2, 2, 1), (7, 3, 3, 2), (6, 12, 3, 2),
                                               (4, 5, 3, 1), (9, 4, 2, 2), (3, 3, 3, 1)])
def test_staged_mrhs_barrier_protocol(ntiles, nrhs, ns, tpt):
    for seed in range(40):
        for land_p in (0.03, 0.3):  # loads that linger, loads that land at once
            _simulate_mrhs(ntiles, nrhs, ns, tpt, seed, land_p)


def test_staged_mrhs_protocol_check_catches_a_ring_deeper_than_nrhs():
    """A planted mistake: three consumer groups for two right-hand sides lets
    a group skip a tile and test a link slot two phases ahead; the simulation
    must notice."""
    caught = 0
    for seed in range(60):
        try:
            _simulate_mrhs(8, 2, 3, 1, seed, 0.03)
        except AssertionError:
            caught += 1
    assert caught > 0


def _simulate_single(ntiles, ns, tpt, seed, land_p=0.3, groups=None):
    """The one-right-hand-side staged kernel: stage g owned by group g (tiles
    k = g, g + ns, ...), one load per tile (links and spinors). `groups` >
    ns plants the first design's mistake (groups sharing stages)."""
    rnd = np.random.default_rng(seed)
    G = groups or ns
    full = [_Barrier(1) for _ in range(ns)]
    empty = [_Barrier(tpt) for _ in range(ns)]
    ready = [_Barrier(1) for _ in range(G * tpt)]
    in_flight = []

    def test(bar, n):
        assert bar.phase in (n, n + 1), (bar.phase, n)
        return (n & 1) != (bar.phase & 1)

    def producer():
        for k in range(ntiles):
            st, n = k % ns, k // ns
            if n >= 1:
                while not test(empty[st], n - 1):
                    yield
            in_flight.append(full[st])
            yield

    def consumer(team, q):
        g = team // tpt
        for m, k in enumerate(range(g, ntiles, G)):
            st = k % ns
            while not test(full[st], k // ns):
                yield
            yield
            if q == 1:
                ready[team].arrive()
            else:
                while not test(ready[team], m):
                    yield
                empty[st].arrive()
            yield

    actors = [producer()] + [consumer(t, q) for t in range(G * tpt) for q in (0, 1)]
    live = list(range(len(actors)))
    steps = 0
    while live or in_flight:
        steps += 1
        assert steps < 200000, "no progress"
        if in_flight and (not live or rnd.random() < land_p):
            in_flight.pop(int(rnd.integers(len(in_flight)))).arrive()
            continue
        if not live:
            continue
        a = live[int(rnd.integers(len(live)))]
        try:
            next(actors[a])
        except StopIteration:
            live.remove(a)


@pytest.mark.parametrize("ntiles,ns,tpt", [(7, 3, 2), (20, 3, 2), (11, 5, 1), (4, 2, 1), (2, 3, 2)])
def test_staged_single_rhs_barrier_protocol(ntiles, ns, tpt):
    for seed in range(40):
        for land_p in (0.03, 0.3):
            _simulate_single(ntiles, ns, tpt, seed, land_p)


def test_staged_protocol_check_catches_groups_sharing_stages():
    """The first design had six groups over two or three stages; the check
    must reject it (the GPU test saw its bounded wait run out)."""
    caught = 0
    for seed in range(60):
        try:
            _simulate_single(16, 2, 1, seed, 0.03, groups=6)
        except AssertionError:
            caught += 1
    assert caught > 0


# ---------------------------------------------------------------------------
# Fused staged M_eo: pair link blocks shared by both hops. Each tile j (R rows
# of one (z, t) plane, T sites of each parity) has one block with the fields
#   eYh | oZ oT oX oY eX eY eZ eT | oYh
# (o/e: links at the tile's odd/even sites, Yh: U_y at the row below the tile).
# A first-hop item (odd output) copies eYh..eY of its block plus eZ of the tile
# in plane z-1 and eT of the tile in plane t-1; a second-hop item (even output)
# copies oX..oYh plus oZ and oT of those tiles. The model below follows the
# kernel's field offsets, copy ranges and consumer indices, and checks every
# link and spinor a consumer reads against the neighbour rule.

def pair_fields(T, lxh):
    f = {"eYh": 0, "oZ": 72 * lxh}
    for a, b in (("oT", "oZ"), ("oX", "oT"), ("oY", "oX"), ("eX", "oY"), ("eY", "eX"), ("eZ", "eY"),
                 ("eT", "eZ"), ("oYh", "eT")):
        f[a] = f[b] + 72 * T
    f["bytes"] = f["oYh"] + 72 * lxh
    return f


def pack_pair_blocks(dims, rows):
    """byte offset in the block array -> (packed field 2 mu + parity, compact
    index) of the link stored there (first float of each link)."""
    lx, ly, lz, lt = dims
    lxh, vh = lx // 2, lx * ly * lz * lt // 2
    T = rows * lxh
    f = pair_fields(T, lxh)
    mem = {}
    for gi in range(vh):
        j, s = divmod(gi, T)
        base = j * f["bytes"]
        for name, fi in (("oX", 1), ("oY", 3), ("oZ", 5), ("oT", 7), ("eX", 0), ("eY", 2), ("eZ", 4), ("eT", 6)):
            mem[base + f[name] + 16 * s] = (fi, gi)
        if s < lxh:
            plane, y0 = divmod(j * rows, ly)
            h = (plane * ly + (y0 - 1) % ly) * lxh + s
            mem[base + f["eYh"] + 16 * s] = (2, h)
            mem[base + f["oYh"] + 16 * s] = (3, h)
    return mem, f


def fs_item(dims, rows, lookahead, q):
    lx, ly, lz, lt = dims
    tpp = ly // rows
    tps = lz * tpp
    k, c = divmod(q, tps)
    kind, t = fused_task(lt, lookahead, k)
    z, yb = divmod(c, tpp)
    y0 = yb * rows
    j = t * tps + c
    jzm = t * tps + ((z - 1) % lz) * tpp + y0 // rows
    jtm = ((t - 1) % lt) * tps + c
    return kind == "B", t, z, y0, j, jzm, jtm


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (8, 4, 6, 6), (8, 8, 8, 8), (16, 2, 4, 4), (12, 6, 4, 8),
                                  (4, 6, 2, 22), (32, 8, 2, 4), (24, 8, 2, 2), (32, 4, 4, 2)])
def test_fused_staged_reads(dims):
    lx, ly, lz, lt = dims
    lxh = lx // 2
    rows = staged_rows(lxh, ly)
    if not rows:
        pytest.skip("not tileable")
    T = rows * lxh
    mem, f = pack_pair_blocks(dims, rows)
    tps = lz * (ly // rows)
    seen = set()
    for q in range(2 * lt * tps):
        b, t, z, y0, j, jzm, jtm = fs_item(dims, rows, 1, q)
        seen.add((b, j))
        # the stage's link region: three copies (destination offset = block offset)
        stage = {}

        def copy(src_tile, off, size):
            for o in range(off, off + size, 16):
                key = src_tile * f["bytes"] + o
                if key in mem:
                    stage[o] = mem[key]

        if not b:
            copy(j, 0, f["eY"] + 72 * T)
            copy(jzm, f["eZ"], 72 * T)
            copy(jtm, f["eT"], 72 * T)
        else:
            copy(j, f["oX"], f["bytes"] - f["oX"])
            copy(jzm, f["oZ"], 72 * T)
            copy(jtm, f["oT"], 72 * T)
        out_parity = 0 if b else 1
        o, e = ("e", "o") if b else ("o", "e")
        fwd = {mu: f[o + "XYZT"[mu]] for mu in range(4)}
        bwd = {mu: f[e + "XYZT"[mu]] for mu in range(4)}
        bwd_halo = f[e + "Yh"]
        boxes, geo = staged_boxes(dims, rows, j)
        assert geo[:3] == (y0, z, t)
        for s in range(T):
            i = j * T + s
            nb, _ = kernel_neighbours(dims, out_parity, i)
            r, xh = divmod(s, lxh)
            for (mu, sgn), region, idx, _d in staged_reads(dims, rows, geo, s, out_parity):
                first, n = boxes[region]
                assert 0 <= idx < n and first + idx == nb[(mu, sgn)]  # spinor read
                if sgn > 0:
                    off, lidx, n_l = fwd[mu], s, T
                elif mu == 0:
                    off, lidx, n_l = bwd[0], r * lxh + (idx - r * lxh), T
                elif mu == 1 and r == 0:
                    off, lidx, n_l = bwd_halo, xh, lxh
                elif mu == 1:
                    off, lidx, n_l = bwd[1], s - lxh, T
                else:
                    off, lidx, n_l = bwd[mu], s, T
                assert 0 <= lidx < n_l
                want = (2 * mu + out_parity, i) if sgn > 0 else (2 * mu + (out_parity ^ 1), nb[(mu, -1)])
                assert stage[off + 16 * lidx] == want, (dims, b, j, s, mu, sgn)
    assert len(seen) == 2 * lt * tps  # every tile once per hop


@pytest.mark.parametrize("lt", [2, 3, 4, 7, 16])
@pytest.mark.parametrize("lookahead", [1, 2, 4])
def test_fused_staged_dependencies_come_first(lt, lookahead):
    """Every second-hop tile's dependencies (all first-hop tiles of slices t-1,
    t, t+1) hold earlier tickets, so the earliest unfinished item never waits."""
    dims = (4, 4, 2, lt)
    rows = staged_rows(2, 4)
    la = max(1, min(lookahead, lt - 1))
    tps = dims[2] * (dims[1] // rows)
    first = {}
    for q in range(2 * lt * tps):
        b, t, *_ = fs_item(dims, rows, la, q)
        if not b:
            first.setdefault(t, []).append(q)
    for q in range(2 * lt * tps):
        b, t, *_ = fs_item(dims, rows, la, q)
        if b:
            for dt in (-1, 0, 1):
                assert max(first[(t + dt) % lt]) < q


@pytest.mark.parametrize("grid", [1, 2, 3, 7, 152])
@pytest.mark.parametrize("lt,lookahead", [(2, 1), (3, 1), (4, 2), (9, 4), (16, 2)])
def test_fused_staged_round_robin_always_progresses(grid, lt, lookahead):
    """The fused staged launch deals the queue round robin: CTA c takes items
    c, c + G, c + 2G, ... in that order and a second-hop item waits until the
    first-hop tiles of slices t-1, t, t+1 are done. Step all CTAs until every
    item is done; some CTA must move at every step (no deadlock), whatever the
    order in which the CTAs run."""
    dims = (4, 4, 2, lt)
    rows = staged_rows(2, 4)
    tps = dims[2] * (dims[1] // rows)
    total = 2 * lt * tps
    items = [fs_item(dims, rows, lookahead, q) for q in range(total)]
    done_a = {t: 0 for t in range(lt)}
    nxt = list(range(grid))  # next item of each CTA
    rng = np.random.default_rng(lt * 100 + grid)
    remaining = total
    while remaining:
        moved = False
        for c in rng.permutation(grid):
            q = nxt[c]
            if q >= total:
                continue
            b, t, *_ = items[q]
            if b and any(done_a[(t + d) % lt] < tps for d in (-1, 0, 1)):
                continue  # waits (bounded in the kernel); other CTAs move
            if not b:
                done_a[t] += 1
            nxt[c] += grid
            remaining -= 1
            moved = True
        assert moved, "no CTA can progress"


def blocked_site_of(dims, b, t):
    """The hop kernels' blocked site order (CTA b, thread t): rows
    (y0 + dy, z0 + dz, t0 + dt) of 2x2x2 blocks, Lx/2 threads per row."""
    lx, ly, lz, lt = dims
    lxh = lx // 2
    hy, hz = ly // 2, lz // 2
    y0, z0, t0 = 2 * (b % hy), 2 * ((b // hy) % hz), 2 * (b // (hy * hz))
    row, xh = divmod(t, lxh)
    return (((t0 + (row >> 2)) * lz + z0 + ((row >> 1) & 1)) * ly + y0 + (row & 1)) * lxh + xh


@pytest.mark.parametrize("dims", [(16, 2, 2, 2), (16, 4, 6, 8), (32, 8, 4, 2), (24, 6, 2, 4), (64, 2, 4, 2)])
def test_blocked_site_order_is_a_permutation(dims):
    """Every site exactly once over the (Ly/2)(Lz/2)(Lt/2) CTAs of 8 Lx/2 threads,
    and each CTA's sites are 8 whole rows forming a 2x2x2 block in (y, z, t)."""
    lx, ly, lz, lt = dims
    lxh, vh = lx // 2, lx * ly * lz * lt // 2
    nb = (ly // 2) * (lz // 2) * (lt // 2)
    seen = []
    for b in range(nb):
        sites = [blocked_site_of(dims, b, t) for t in range(8 * lxh)]
        rows = sorted({s // lxh for s in sites})
        assert len(rows) == 8 and all(len([s for s in sites if s // lxh == r]) == lxh for r in rows)
        ys = {r % ly for r in rows}
        zs = {(r // ly) % lz for r in rows}
        ts = {r // (ly * lz) for r in rows}
        assert len(ys) == len(zs) == len(ts) == 2
        seen += sites
    assert sorted(seen) == list(range(vh))
