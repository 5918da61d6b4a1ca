"""The library's static task schedules (setup.cpp), checked on the CPU through
the host harness:

* race check: within one launch (a step: its tile tasks run as CTAs in any
  order) and between stream groups (no ordering at all) no two tasks touch a
  byte that one of them writes;
* host execution: the schedule run task by task with the tile kernels'
  semantics (groups interleaved at random, the tasks of a step shuffled)
  reproduces the block Cholesky factor, the block inverses and the block
  triangular solves of a random SPD block-tridiagonal matrix (numpy);
* a planted scheduling mistake (two dependent steps merged into one launch,
  two subdomains scattering into one buffer) is reported by the race check.

Covers the right- and left-looking factorisations, 1 to 32 stream groups, the
FP64 and FP32 (mixed) schedules, PST- and KB-wide solves, memory-bounded
waves and the coarse-problem schedules (Sec. 4.5's direct subdomain solver,
restated as layer-block Cholesky)."""
import numpy as np
import pytest

from tests.host import hostcheck as hc

pytestmark = pytest.mark.skipif(hc.cuda_include() is None, reason="host harness needs the CUDA headers")


def _cfg(name):
    from workloads import get_config
    return get_config(name)


def _mv(hs, members, width, rng, fill=True):
    out = [None] * hs.N
    for j in members:
        n = hs.sub(j)["nfull"]
        out[j] = rng.standard_normal((n, width)) if fill else np.zeros((n, width))
    return out


def _width(which):
    return hc.KB if which in (hc.SC_SOLVE_K8, hc.SC_SOLVE_A8) else hc.PST


@pytest.mark.parametrize("name", ["t2", "s1"])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("left", [False, True])
@pytest.mark.parametrize("groups", [(16, 16), (1, 1), (32, 32), (3, 5)])
def test_schedules_are_race_free(name, mixed, left, groups):
    _race_free(name, mixed, left, groups)


@pytest.mark.parametrize("name", ["t4", "s2"])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("left", [False, True])
@pytest.mark.parametrize("groups", [(16, 16), (3, 5)])
def test_schedules_are_race_free_multi_tile(name, mixed, left, groups):
    """Larger layers (several 64-row tiles per layer block, 8 and 12 subdomains),
    right- and left-looking, even and uneven stream-group splits."""
    _race_free(name, mixed, left, groups)


def _race_free(name, mixed, left, groups):
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=mixed)
    assert hs.status == 0, hs.error
    assert hs.plan_waves(1e15) == 1
    hs.build_wave(0, groups[0], groups[1], left)
    members = hs.members(0)
    ng, nsteps, ntasks = hs.shape(hc.SC_FACTOR)
    assert ng == groups[0] and ntasks > 0
    n, msg = hs.race(hc.SC_FACTOR)
    assert n == 0, msg
    rng = np.random.default_rng(0)
    for which in hc.SOLVES:
        g, _, nt = hs.shape(which)
        assert g == groups[1] and nt > 0
        src = _mv(hs, members, _width(which), rng)
        dst = _mv(hs, members, _width(which), rng)
        for d, add in ((dst, False), (dst, True), (src, False)):     # separate buffers, accumulate, in place
            n, msg = hs.race(which, src, d, scatter_add=add)
            assert n == 0, (which, msg)


def _fill_spd(hs, j, matrix, rng):
    """Random SPD block-tridiagonal matrix in subdomain j's layer blocks (padding
    rows identity, never-read upper tiles NaN); returns the dense compact matrix."""
    s = hs.sub(j)
    n = s["nK"] if matrix == "K" else s["nA"]
    D, E, Li = hs.blocks(j, matrix)
    nz, b = D.shape[0], D.shape[1]
    T = b // hc.TILE
    upper = np.zeros((b, b), dtype=bool)
    for ti in range(T):
        for tj in range(ti + 1, T):
            upper[ti * hc.TILE:(ti + 1) * hc.TILE, tj * hc.TILE:(tj + 1) * hc.TILE] = True
    M = np.zeros((nz * n, nz * n))
    for l in range(nz):
        S = rng.uniform(-1, 1, (n, n)) / np.sqrt(n)
        S = (S + S.T) / 2 + 6.0 * np.eye(n)
        blk = np.eye(b)
        blk[:n, :n] = S
        blk[upper] = np.nan
        D[l] = blk
        M[l * n:(l + 1) * n, l * n:(l + 1) * n] = S
    for l in range(nz - 1):
        blk = np.zeros((b, b))
        blk[:n, :n] = rng.uniform(-1, 1, (n, n)) / np.sqrt(n)
        E[l] = blk
        M[(l + 1) * n:(l + 2) * n, l * n:(l + 1) * n] = blk[:n, :n]
        M[l * n:(l + 1) * n, (l + 1) * n:(l + 2) * n] = blk[:n, :n].T
    Li[:] = np.nan
    return M, n, upper


def _check_factor(hs, j, matrix, M, n, upper, tol):
    D, E, Li = hs.blocks(j, matrix)
    nz = D.shape[0]
    L = np.linalg.cholesky(M)
    scale = np.abs(L).max()
    low = ~upper
    for l in range(nz):
        Ll = L[l * n:(l + 1) * n, l * n:(l + 1) * n]
        got = np.where(low, D[l].astype(np.float64), 0.0)
        assert np.isfinite(got).all()
        np.testing.assert_allclose(np.tril(got[:n, :n]), Ll, atol=tol * scale, rtol=0)
        assert np.allclose(np.triu(got[:n, :n], 1), 0.0)
        inv = np.linalg.inv(Ll)
        gi = np.where(low, Li[l].astype(np.float64), np.nan)[:n, :n]
        np.testing.assert_allclose(np.tril(gi), inv, atol=tol * np.abs(inv).max(), rtol=0)
        if l + 1 < nz:
            np.testing.assert_allclose(E[l][:n, :n].astype(np.float64), L[(l + 1) * n:(l + 2) * n, l * n:(l + 1) * n],
                                       atol=tol * scale, rtol=0)


def _check_solve(hs, j, matrix, M, n, src, dst0, dst, gather_neg, scatter_add, tol):
    s = hs.sub(j)
    a = hs.arrays(j)
    mp = (a["mapK"] if matrix == "K" else a["mapA"])[:n]
    nz, npl = s["nzn"], s["npl"]
    rows = np.concatenate([l * 3 * npl + mp for l in range(nz)])
    rhs = (-1.0 if gather_neg else 1.0) * src[rows]
    x = np.linalg.solve(M, rhs)
    exp = dst0.copy()
    exp[rows] = (exp[rows] if scatter_add else 0.0) + x
    keep = np.ones(len(dst), dtype=bool)
    keep[rows] = False
    np.testing.assert_array_equal(dst[keep], dst0[keep])      # rows outside the matrix untouched
    np.testing.assert_allclose(dst[rows], exp[rows], atol=tol * np.abs(x).max(), rtol=0)


@pytest.mark.parametrize("name, mixed, left, groups", [
    ("t2", False, False, (16, 16)),
    ("t2", False, True, (3, 5)),
    ("t2", True, True, (16, 16)),
    ("s1", False, True, (32, 4)),
    ("s1", True, False, (1, 1)),
    ("c1", False, False, (16, 16)),
])
def test_schedules_execute_to_the_block_cholesky(name, mixed, left, groups):
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=mixed)
    assert hs.plan_waves(1e15) == 1
    hs.build_wave(0, groups[0], groups[1], left)
    members = hs.members(0)
    rng = np.random.default_rng(1)
    mats = {}
    for j in members:
        for matrix in "KA":
            mats[j, matrix] = _fill_spd(hs, j, matrix, rng)
    assert hs.run_factor(seed=7) == 0
    tol = 2e-4 if mixed else 1e-11
    for (j, matrix), (M, n, upper) in mats.items():
        _check_factor(hs, j, matrix, M, n, upper, tol)
    for which, matrix in ((hc.SC_SOLVE_K, "K"), (hc.SC_SOLVE_A, "A"), (hc.SC_SOLVE_K8, "K"), (hc.SC_SOLVE_A8, "A")):
        w = _width(which)
        for gather_neg, scatter_add in ((False, False), (True, True)):
            src = _mv(hs, members, w, rng)
            dst0 = _mv(hs, members, w, rng)
            dst = [None if d is None else d.copy() for d in dst0]
            hs.run_solve(which, src, dst, gather_neg, scatter_add, seed=11)
            for j in members:
                M, n, _ = mats[j, matrix]
                _check_solve(hs, j, matrix, M, n, src[j], dst0[j], dst[j], gather_neg, scatter_add, tol)


@pytest.mark.parametrize("name, left, window", [("t2", False, 1), ("t2", True, 7), ("s1", False, 64),
                                                ("c1", True, 3)])
def test_persistent_factorisation_order(name, left, window):
    """The persistent FP32 factorisation's ticket order (every task once, one
    dependency group per chain) run as `window` resident CTAs that take tickets
    in order and start a task once the previous step of its chain is complete:
    it never deadlocks (window 1 means the order itself is topological) and
    reproduces the block Cholesky factor and inverses."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=True)
    assert hs.plan_waves(1e15) == 1
    hs.set_persistent(True)
    hs.build_wave(0, 16, 16, left)
    members = hs.members(0)
    assert hs.persistent_tasks() > 0
    rng = np.random.default_rng(2)
    mats = {}
    for j in members:
        for matrix in "KA":
            mats[j, matrix] = _fill_spd(hs, j, matrix, rng)
    assert hs.run_factor_persistent(window, seed=5) == 0
    for (j, matrix), (M, n, upper) in mats.items():
        _check_factor(hs, j, matrix, M, n, upper, 2e-4)
    hs.close()


def test_waves_schedule_only_their_members():
    """With a budget of about a third, each wave's schedules factorise exactly
    its members (the others' blocks are left alone; they share the pool)."""
    cfg = _cfg("s2")
    hs = hc.HostSetup(cfg)
    sizes = np.array([hs.sub_bytes(j) for j in range(hs.N)])
    nw = hs.plan_waves(sizes.sum() // 3)
    assert nw >= 3
    rng = np.random.default_rng(2)
    for w in range(nw):
        hs.build_wave(w, 16, 16, left=(w % 2 == 1))
        members = hs.members(w)
        n, msg = hs.race(hc.SC_FACTOR)
        assert n == 0, msg
        if w != nw - 1:
            continue
        mats = {(j, m): _fill_spd(hs, j, m, rng) for j in members for m in "KA"}
        assert hs.run_factor(seed=w) == 0
        for (j, m), (M, n, upper) in mats.items():
            _check_factor(hs, j, m, M, n, upper, 1e-11)
        src = _mv(hs, members, hc.KB, rng)
        dst = _mv(hs, members, hc.KB, rng, fill=False)
        others = [None if j in members else np.full((hs.sub(j)["nfull"], hc.KB), 5.0) for j in range(hs.N)]
        src2 = [s if s is not None else o for s, o in zip(src, others)]
        dst2 = [d if d is not None else o.copy() for d, o in zip(dst, others)]
        hs.run_solve(hc.SC_SOLVE_K8, src2, dst2, seed=3)
        for j in range(hs.N):
            if j not in members:
                assert (dst2[j] == 5.0).all()
            else:
                M, n, _ = mats[j, "K"]
                _check_solve(hs, j, "K", M, n, src[j], np.zeros_like(dst2[j]), dst2[j], False, False, 1e-11)


@pytest.mark.parametrize("tiles", [4, 20])
def test_coarse_schedules(tiles):
    """The coarse Galerkin matrix: one dense block of NcPad rows factorised by the
    same tile tasks and solved by one forward and one backward sweep; with 20
    tiles the block inverse's long rows (more than 8 tile products) run as
    partial sums into scratch tiles plus a final task through the identity
    strip."""
    cfg = _cfg("t2")
    hs = hc.HostSetup(cfg)
    rng = np.random.default_rng(3)
    b = tiles * hc.TILE
    G = rng.standard_normal((b, b)) / np.sqrt(b)
    A = G @ G.T + 0.5 * np.eye(b)
    AH = A.copy()
    AHinv = np.full((b, b), np.nan)
    bH = rng.standard_normal((b, hc.PST))
    rH, yH, cH = (np.zeros((b, hc.PST)) for _ in range(3))
    hs.build_coarse(b, AH, AHinv, bH, rH, yH, cH)
    for which in (hc.SC_COARSE_FACTOR, hc.SC_COARSE_SOLVE):
        n, msg = hs.race(which)
        assert n == 0, msg
    assert hs.run_factor(seed=5, coarse=True) == 0
    L = np.linalg.cholesky(A)
    np.testing.assert_allclose(np.tril(AH), L, atol=1e-12 * np.abs(L).max(), rtol=0)
    np.testing.assert_allclose(np.tril(AHinv), np.linalg.inv(L), rtol=0, atol=1e-11 * np.abs(np.linalg.inv(L)).max())
    hs.run_solve(hc.SC_COARSE_SOLVE, None, None, seed=5)
    np.testing.assert_allclose(cH, np.linalg.solve(A, bH), rtol=0, atol=1e-11 * np.abs(cH).max())


def test_not_positive_definite_tile_is_reported():
    cfg = _cfg("t1")
    hs = hc.HostSetup(cfg)
    hs.plan_waves(1e15)
    hs.build_wave(0, 16, 16)
    rng = np.random.default_rng(4)
    for j in hs.members(0):
        for m in "KA":
            _fill_spd(hs, j, m, rng)
    D, _, _ = hs.blocks(hs.members(0)[0], "K")
    D[0][3, 3] = -1.0
    assert hs.run_factor(seed=1) >= 1


def test_race_check_reports_planted_mistakes():
    cfg = _cfg("t2")
    hs = hc.HostSetup(cfg)
    hs.plan_waves(1e15)
    hs.build_wave(0, 1, 1, left=False)
    members = hs.members(0)
    # POTRF of column 0 and the TRMM that reads its inverse in one launch
    assert hs.merge_steps(hc.SC_FACTOR, 0, 1) == 0
    n, msg = hs.race(hc.SC_FACTOR)
    assert n > 0 and "overlap" in msg
    # forward-sweep gather and triangular solve of a layer in one launch
    rng = np.random.default_rng(5)
    src = _mv(hs, members, hc.KB, rng)
    dst = _mv(hs, members, hc.KB, rng)
    assert hs.race(hc.SC_SOLVE_K8, src, dst)[0] == 0
    assert hs.merge_steps(hc.SC_SOLVE_K8, 0, 0) == 0
    assert hs.race(hc.SC_SOLVE_K8, src, dst)[0] > 0
    # two subdomains (in different stream groups) scattering into one buffer
    hs.build_wave(0, 16, 16)
    src = _mv(hs, members, hc.PST, rng)
    dst = _mv(hs, members, hc.PST, rng)
    assert hs.race(hc.SC_SOLVE_K, src, dst)[0] == 0
    a, b = members[0], members[1]
    big = dst[a] if dst[a].shape[0] >= dst[b].shape[0] else dst[b]
    dst[a] = dst[b] = big
    n, msg = hs.race(hc.SC_SOLVE_K, src, dst)
    assert n > 0 and "group" in msg, msg


@pytest.mark.parametrize("name", ["t2", "s1", "c1"])
@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("left", [False, True])
def test_vector_load_preconditions(name, mixed, left):
    """The tile kernels load operands as 16-byte vectors (float4 / double2,
    cp.async of 16 bytes): every operand pointer and leading dimension of every
    task is 16-byte aligned, every inner dimension a multiple of the vector
    width, and the schedules' summary flags (all K % 32 == 0 for the FP32 GEMM
    fast path, all K % 64 == 0 for the cp.async solve ring, the largest K for
    shared-memory sizing) are true to their tasks; for every wave of a split
    pool as well."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=mixed)
    sizes = np.array([hs.sub_bytes(j) for j in range(hs.N)])
    for budget in (1e15, max(sizes.max(), sizes.sum() // 2)):
        nw = hs.plan_waves(budget)
        for w in range(nw):
            hs.build_wave(w, 16, 16, left)
            for which in (hc.SC_FACTOR,) + hc.SOLVES:
                n, msg = hs.align_check(which)
                assert n == 0, (which, msg)
    b = 3 * hc.TILE
    bufs = [np.zeros((b, b)), np.zeros((b, b))] + [np.zeros((b, hc.PST)) for _ in range(4)]
    hs.build_coarse(b, *bufs)
    for which in (hc.SC_COARSE_FACTOR, hc.SC_COARSE_SOLVE):
        assert hs.align_check(which) == (0, "")


def test_vector_load_check_reports_misalignment():
    cfg = _cfg("t2")
    hs = hc.HostSetup(cfg)
    b = 3 * hc.TILE
    off = np.zeros(b * b + 1)[1:].reshape(b, b)          # 8 bytes past a 16-byte boundary
    assert off.ctypes.data % 16 == 8
    bufs = [off, np.zeros((b, b))] + [np.zeros((b, hc.PST)) for _ in range(4)]
    hs.build_coarse(b, *bufs)
    n, msg = hs.align_check(hc.SC_COARSE_FACTOR)
    assert n > 0 and "misaligned" in msg


def test_algorithmic_flops_do_not_exceed_the_executed_ones():
    """The bench's factorisation roofline divides the algorithmic flops of a
    block-tridiagonal Cholesky (per matrix, n^3/3 per layer plus 2 n^3 between
    layers, n the unpadded layer size) by the measured time.  The tile tasks of
    the schedules execute more: the explicit inverses of the diagonal factors
    (n^3/3 per layer), 64-row padding and whole diagonal tiles.  On the full c2
    beam the FP32 tasks execute 1.21 times the count with the inverses and
    1.38 times the algorithmic one, the same for both schedules; the FP64
    kernel skips the zero blocks of the triangular operand of its TRMM tasks
    and post-multiplications and the blocks above the diagonal of diagonal
    output tiles (10 of 16 blocks computed), 1.27 times the algorithmic count.  Either way the
    reported fraction of peak understates the rate of the tile kernel."""
    cfg = _cfg("c2")
    found = {}
    for mixed in (False, True):
        ratios, ratios_inv = set(), set()
        hs = hc.HostSetup(cfg, mixed=mixed)
        assert hs.plan_waves(1e18) == 1
        alg = alg_inv = 0.0
        for j in range(hs.N):
            s = hs.sub(j)
            for n in (s["nK"], s["nA"]):
                alg += s["nzn"] * n ** 3 / 3.0 + (s["nzn"] - 1) * 2.0 * n ** 3
                alg_inv += s["nzn"] * 2.0 * n ** 3 / 3.0 + (s["nzn"] - 1) * 2.0 * n ** 3
        for left in (False, True):
            hs.build_wave_virtual(0, 16, 16, left)
            ratios.add(round(hs.factor_task_flops() / alg, 6))
            ratios_inv.add(round(hs.factor_task_flops() / alg_inv, 6))
        assert len(ratios) == 1 and len(ratios_inv) == 1
        found[mixed] = (ratios.pop(), ratios_inv.pop())
    r32, ri32 = found[True]
    r64, ri64 = found[False]
    assert 1.15 < ri32 < 1.25 and 1.25 < r32 < 1.40, found
    assert 1.0 < r64 < r32 and 1.26 < r64 < 1.31, found


@pytest.mark.parametrize("name", ["t2", "s2", "c2", "c4"])
def test_tma_solve_preconditions(name):
    """Every FP32 8-column solve task with an inner dimension satisfies the
    slab conditions the TMA-filled solve ring checks on the device (its error
    path never fires on the library's own schedules), on full-size schedules
    built on a virtual pool."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=True)
    assert hs.plan_waves(1e18) == 1
    hs.build_wave_virtual(0, 16, 4, left=False)
    for which in (hc.SC_SOLVE_K8, hc.SC_SOLVE_A8):
        n, msg = hs.tma_check(which)
        assert n == 0, (which, msg)
    hs.close()


@pytest.mark.parametrize("name", ["c2", "c4"])
@pytest.mark.parametrize("mixed", [False, True])
def test_vector_load_preconditions_at_full_size(name, mixed):
    """The same preconditions on the full-size schedules: the c2 beam (32
    subdomains, ~0.96M tile tasks) and the c4 spar (256 uneven subdomains,
    ~12.7M tile tasks), built on a virtual pool."""
    cfg = _cfg(name)
    hs = hc.HostSetup(cfg, mixed=mixed)
    assert hs.plan_waves(1e18) == 1
    hs.build_wave_virtual(0, 16, 16, left=True)
    for which in (hc.SC_FACTOR,) + hc.SOLVES:
        n, msg = hs.align_check(which)
        assert n == 0, (which, msg)
