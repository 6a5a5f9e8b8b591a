"""GPU parity of the variable-diffusivity path: single steps, batches of
independent problems and the checkpointed adjoint, against the FP64 oracle.

Tolerance: norm-wise relative 1e-12 for fields, 1e-11 for gradients (the
kernels use the algebraically equal form m*u + sum w_f u_b with fused
multiply-adds, the oracle the flux differences with separate roundings: they
differ by a few ulps per step; the gradient sums products of differences and
loses one more digit).  Schedules (plain / graph / fused, checkpoint
interval) must agree bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1810_11482_b300 import hxc, synth

pytestmark = pytest.mark.gpu
TOL = 1e-12
TOLG = 1e-11


@pytest.fixture(scope="module")
def dev():
    devs = hxc.get_all_devices(2, 0)
    assert devs
    return devs[0]


def up(dev, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = dev.buffer(max(a.nbytes, 8))
    b.write(a).get()
    return b


def down(b, shape):
    out = np.empty(shape, dtype=np.float64)
    b.read_sync(out)
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------- single steps

@pytest.mark.parametrize("ny,nx", [(16, 12), (33, 70), (1, 9), (64, 64)])
def test_varcoef_launch_steps_vs_oracle(dev, ny, nx):
    kap = synth.uniform(400 + nx, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    u0 = synth.uniform(401 + nx, ny * nx).reshape(ny, nx)
    c = 0.9 / (4 * kap.max())
    bk, bu, bt = up(dev, kap), up(dev, u0), dev.buffer(u0.nbytes)
    cur, nxt = bu, bt
    for step in range(1, 8):
        dev.launch(hxc.HXC_K_VARCOEF2D, hxc.hxc_varcoef2d_args(cur.h, nxt.h, bk.h, ny, nx, c)).get()
        cur, nxt = nxt, cur
        assert rel(down(cur, (ny, nx)), oracle.varcoef2d(u0, kap, c, step)) <= TOL
    # the precomputed-coefficient forward run gives the same bits
    out = dev.buffer(u0.nbytes)
    f, st = hxc.varcoef_forward_run(dev, up(dev, u0), bk, ny, nx, c, 7, out)
    f.get()
    assert np.array_equal(down(out, (ny, nx)), down(cur, (ny, nx)))
    assert st.kernel_launches == 8


def test_varcoef_forward_rejects_aliasing(dev):
    b = up(dev, np.zeros((4, 4)))
    k = up(dev, np.ones((4, 4)))
    with pytest.raises(hxc.HxcError):
        hxc.varcoef_forward_run(dev, b, k, 4, 4, 0.1, 3, b)


# ----------------------------------------------------------------- batches

def run_batch(dev, sides, kap, u0, cs, steps, mode):
    bu, bk = up(dev, u0), up(dev, kap)
    f, st = hxc.varcoef_batch_run(dev, bu, bk, sides, cs, steps, mode)
    f.get()
    return down(bu, u0.shape), st


def test_batch_small_vs_oracle_all_modes(dev):
    sides, offs, kap, u0, cs = synth.batch_input(nprob=37, seed=410, smin=1, smax=70)
    for steps in (0, 1, 2, 9):
        want = oracle.varcoef2d_batch(u0, kap, sides, offs, cs, steps)
        outs = {}
        for mode in ("plain", "graph", "fused"):
            got, st = run_batch(dev, sides, kap, u0, cs, steps, mode)
            assert rel(got, want) <= TOL, (steps, mode)
            outs[mode] = got
        assert np.array_equal(outs["plain"], outs["graph"])
        assert np.array_equal(outs["plain"], outs["fused"])


def test_batch_smem_resident_problems_bit_identical(dev):
    """Problems up to the side set by batch.smem_side run with both fields
    in shared memory for the whole run: the persistent launch gives the
    same bits for every threshold (none, some, all problems resident), for
    even and odd step counts, as the per-step schedule."""
    sides = np.array([1, 2, 31, 32, 33, 40, 59, 64, 70, 97, 119, 120, 150, 7, 64, 1], dtype=np.int64)
    sides, offs, kap, u0, cs = synth.batch_input(seed=411, sides=sides)
    old = hxc.tune_get("batch.smem_side")
    try:
        for steps in (1, 6, 9):
            want = oracle.varcoef2d_batch(u0, kap, sides, offs, cs, steps)
            ref, _ = run_batch(dev, sides, kap, u0, cs, steps, "graph")
            assert rel(ref, want) <= TOL
            for side in (0, 32, 59, 119):
                hxc.tune_set("batch.smem_side", side)
                got, st = run_batch(dev, sides, kap, u0, cs, steps, "fused")
                assert st.kernel_launches == 1
                assert np.array_equal(got, ref), (steps, side)
    finally:
        hxc.tune_set("batch.smem_side", old)


def test_batch_full_config(dev):
    """4096 problems, sides log-uniform in [32, 1024], kappa U[0.5, 1.5),
    c at 0.9 of the stability limit, 50 steps: fused (one persistent launch)
    and graph (batched per-step launches) bit-identical; every problem of the
    batch against the oracle (its OpenMP build: problems spread over the host
    threads)."""
    sides, offs, kap, u0, cs = synth.batch_input(nprob=4096, seed=4)
    steps = 50
    fused, st = run_batch(dev, sides, kap, u0, cs, steps, "fused")
    assert st.kernel_launches == 1
    graph, st = run_batch(dev, sides, kap, u0, cs, steps, "graph")
    assert np.array_equal(fused, graph)
    want = oracle.varcoef2d_batch(u0, kap, sides, offs, cs, steps, omp=True)
    for p in range(sides.size):
        o, s = offs[p], sides[p]
        assert rel(fused[o:o + s * s], want[o:o + s * s]) <= TOL, p
    assert np.all(np.isfinite(fused)) and fused.min() >= 0.0 and fused.max() <= 1.0


# ----------------------------------------------------------------- adjoint

def adjoint(dev, u0, kap, lamT, c, steps, every=0, mode="fused"):
    ny, nx = u0.shape
    bu, bk, bl = up(dev, u0), up(dev, kap), up(dev, lamT)
    gk, gu, uT = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    f, st = hxc.varcoef_adjoint_run(dev, bu, bk, bl, ny, nx, c, steps, gk, gu, uT, every, mode)
    f.get()
    return down(gk, u0.shape), down(gu, u0.shape), down(uT, u0.shape), st


def test_adjoint_small_vs_oracle_and_schedules(dev):
    ny, nx, steps, c = 16, 12, 7, 0.15
    kap = synth.uniform(420, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    u0 = synth.uniform(421, ny * nx).reshape(ny, nx)
    tgt = synth.uniform(422, ny * nx).reshape(ny, nx)
    loss, ogk, ogu = oracle.varcoef2d_adjoint(u0, kap, tgt, c, steps)
    uT = oracle.varcoef2d(u0, kap, c, steps)
    lamT = 2.0 * (uT - tgt)  # seed from the oracle's final state
    ref = None
    for every in (0, 1, 2, 3, 7, 9):
        for mode in ("plain", "graph", "fused"):
            gk, gu, guT, st = adjoint(dev, u0, kap, lamT, c, steps, every, mode)
            assert rel(guT, uT) <= TOL
            assert rel(gk, ogk) <= TOLG and rel(gu, ogu) <= TOLG, (every, mode)
            if ref is None:
                ref = (gk, gu)
            assert np.array_equal(gk, ref[0]) and np.array_equal(gu, ref[1]), (every, mode)


def test_checkpoint_tape_matches_adjoint_run(dev):
    """A forward run that keeps its checkpoints (hxc_varcoef_forward_tape)
    gives the forward run's final state and, as checkpoint k, the state after
    k * every steps; the adjoint from that tape gives the bits of the adjoint
    run that does its own forward pass, for every checkpoint interval and
    mode; a tape that is too small is rejected."""
    ny, nx, c = 18, 13, 0.15
    kap = synth.uniform(423, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    u0 = synth.uniform(424, ny * nx).reshape(ny, nx)
    lamT = synth.uniform(427, ny * nx, lo=-1, hi=1).reshape(ny, nx)
    bu, bk, bl = up(dev, u0), up(dev, kap), up(dev, lamT)
    for steps in (0, 1, 7, 10):
        want_uT = dev.buffer(u0.nbytes)
        hxc.varcoef_forward_run(dev, bu, bk, ny, nx, c, steps, want_uT)[0].get()
        want_uT = down(want_uT, u0.shape)
        for every in (0, 1, 2, 3, 7, 9):
            ns = hxc.varcoef_tape_states(steps, every)
            e = every or max(1, int(np.ceil(np.sqrt(max(1, steps)))))
            assert ns == (max(1, -(-steps // e)) if steps else 1)
            tape, uT = dev.buffer(ns * u0.nbytes), dev.buffer(u0.nbytes)
            hxc.varcoef_forward_tape(dev, bu, bk, ny, nx, c, steps, uT, tape, every)[0].get()
            assert np.array_equal(down(uT, u0.shape), want_uT), (steps, every)
            tp = down(tape, (ns, ny, nx))
            for kk in range(ns):
                ref = dev.buffer(u0.nbytes)
                hxc.varcoef_forward_run(dev, bu, bk, ny, nx, c, kk * e, ref)[0].get()
                assert np.array_equal(tp[kk], down(ref, u0.shape)), (steps, every, kk)
            for mode in ("plain", "graph", "fused"):
                gk, gu, _, _ = adjoint(dev, u0, kap, lamT, c, steps, every, mode)
                tk, tu = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
                hxc.varcoef_adjoint_tape(dev, tape, bk, bl, ny, nx, c, steps, tk, tu, every,
                                         mode)[0].get()
                assert np.array_equal(down(tk, u0.shape), gk), (steps, every, mode)
                assert np.array_equal(down(tu, u0.shape), gu), (steps, every, mode)
    small = dev.buffer(u0.nbytes)
    with pytest.raises(hxc.HxcError):
        hxc.varcoef_forward_tape(dev, bu, bk, ny, nx, c, 10, dev.buffer(u0.nbytes), small, 3)
    # outputs that would overwrite the tape while the run reads it are rejected
    big = dev.buffer(4 * u0.nbytes)
    hxc.varcoef_forward_tape(dev, bu, bk, ny, nx, c, 10, dev.buffer(u0.nbytes), big, 3)[0].get()
    inside = dev.wrap(big.ptr + u0.nbytes, u0.nbytes)
    with pytest.raises(hxc.HxcError):
        hxc.varcoef_adjoint_tape(dev, big, bk, bl, ny, nx, c, 10, inside, dev.buffer(u0.nbytes), 3)
    with pytest.raises(hxc.HxcError):
        hxc.varcoef_adjoint_tape(dev, small, bk, bl, ny, nx, c, 10, dev.buffer(u0.nbytes),
                                 dev.buffer(u0.nbytes), 3)


def test_adjoint_zero_steps(dev):
    u0 = synth.uniform(425, 30).reshape(5, 6)
    kap = np.ones((5, 6))
    lam = synth.uniform(426, 30).reshape(5, 6)
    gk, gu, uT, _ = adjoint(dev, u0, kap, lam, 0.1, 0)
    assert np.array_equal(gu, lam) and np.all(gk == 0.0) and np.array_equal(uT, u0)


def test_adjoint_launch_kernel_matches_fused(dev):
    """The hxc_launch adjoint kernel (coefficients on the fly) gives the same
    bits as the fused driver for one step."""
    ny, nx, c = 20, 17, 0.15
    kap = synth.uniform(430, ny * nx, lo=0.5, hi=1.5).reshape(ny, nx)
    u0 = synth.uniform(431, ny * nx).reshape(ny, nx)
    lam = synth.uniform(432, ny * nx, lo=-1, hi=1).reshape(ny, nx)
    gk, gu, _, _ = adjoint(dev, u0, kap, lam, c, 1)
    bl, bo, bu, bk = up(dev, lam), dev.buffer(u0.nbytes), up(dev, u0), up(dev, kap)
    bg = up(dev, np.zeros_like(u0))
    dev.launch(hxc.HXC_K_ADJOINT2D, hxc.hxc_adjoint2d_args(bl.h, bo.h, bu.h, bk.h, bg.h, ny, nx, c)).get()
    assert np.array_equal(down(bo, u0.shape), gu)
    assert np.array_equal(down(bg, u0.shape), gk)


def test_adjoint_medium_vs_oracle(dev):
    n, steps, c = 96, 40, 0.15
    kref, kap, _, _ = synth.adjoint_input(n)
    u0 = synth.bumps2d(n, n, seed=7, nbumps=6, sigma=0.08)
    tgt = oracle.varcoef2d(u0, kref, c, steps)
    loss, ogk, ogu = oracle.varcoef2d_adjoint(u0, kap, tgt, c, steps)
    uT = oracle.varcoef2d(u0, kap, c, steps)
    gk, gu, guT, _ = adjoint(dev, u0, kap, 2.0 * (uT - tgt), c, steps)
    assert rel(gk, ogk) <= TOLG and rel(gu, ogu) <= TOLG
    # loss through the squared-error kernel
    bu, bt, bl, bls = up(dev, guT), up(dev, tgt), dev.buffer(u0.nbytes), dev.buffer(8)
    hxc.sqerr_seed(dev, bu, bt, bl, bls, n * n).get()
    assert abs(down(bls, 1)[0] - loss) <= 1e-12 * loss
    assert rel(down(bl, u0.shape), 2.0 * (uT - tgt)) <= 1e-12


def test_adjoint_full_config_properties(dev):
    """2048^2, 500 steps, c = 0.15, checkpoints every ceil(sqrt(500)) = 23
    steps: gradient identical to the store-all schedule; dL/du0 identical to
    the forward operator applied to 2 (u^T - u_tgt); central differences on
    the 32 random joint directions (dkappa, du0) agree with the adjoint's
    directional derivatives (relative 1e-6 for kappa, 1e-9 for u0, where the
    loss is quadratic and central differences are exact up to rounding)."""
    n, steps, c = 2048, 500, 0.15
    kref, kap, u0, _ = synth.adjoint_input(n)
    bu0, bkr, bk = up(dev, u0), up(dev, kref), up(dev, kap)
    tgt = dev.buffer(u0.nbytes)
    hxc.varcoef_forward_run(dev, bu0, bkr, n, n, c, steps, tgt)[0].get()
    uT = dev.buffer(u0.nbytes)
    hxc.varcoef_forward_run(dev, bu0, bk, n, n, c, steps, uT)[0].get()
    lam, loss_b = dev.buffer(u0.nbytes), dev.buffer(8)
    hxc.sqerr_seed(dev, uT, tgt, lam, loss_b, n * n).get()
    L0 = down(loss_b, 1)[0]
    gk, gu = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    f, st = hxc.varcoef_adjoint_run(dev, bu0, bk, lam, n, n, c, steps, gk, gu, None, 0, "fused")
    f.get()
    gk_h, gu_h = down(gk, u0.shape), down(gu, u0.shape)
    # store-all schedule
    gk2, gu2 = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    hxc.varcoef_adjoint_run(dev, bu0, bk, lam, n, n, c, steps, gk2, gu2, None, 1, "fused")[0].get()
    assert np.array_equal(down(gk2, u0.shape), gk_h) and np.array_equal(down(gu2, u0.shape), gu_h)
    # the training-step form: forward with a checkpoint tape, adjoint from it
    tape = dev.buffer(hxc.varcoef_tape_states(steps) * u0.nbytes)
    uT2, gk3, gu3 = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)
    hxc.varcoef_forward_tape(dev, bu0, bk, n, n, c, steps, uT2, tape)[0].get()
    assert np.array_equal(down(uT2, u0.shape), down(uT, u0.shape))
    hxc.varcoef_adjoint_tape(dev, tape, bk, lam, n, n, c, steps, gk3, gu3)[0].get()
    assert np.array_equal(down(gk3, u0.shape), gk_h) and np.array_equal(down(gu3, u0.shape), gu_h)
    del tape, uT2, gk3, gu3
    # dL/du0 = A^steps lambda^T (symmetric step matrix, same kernel)
    fw = dev.buffer(u0.nbytes)
    hxc.varcoef_forward_run(dev, lam, bk, n, n, c, steps, fw)[0].get()
    assert np.array_equal(down(fw, u0.shape), gu_h)
    del gk2, gu2, fw

    bkx, bux, out = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(u0.nbytes)

    def loss_at(kappa, uinit):
        bkx.write(np.ascontiguousarray(kappa)).get()
        bux.write(np.ascontiguousarray(uinit)).get()
        hxc.varcoef_forward_run(dev, bux, bkx, n, n, c, steps, out)[0].get()
        hxc.sqerr_seed(dev, out, tgt, None, loss_b, n * n).get()
        return down(loss_b, 1)[0]

    eps_k, eps_u = 1e-4 * np.abs(kap).max(), 1e-3
    nk, ngu = np.linalg.norm(gk_h), np.linalg.norm(gu_h)
    worst_k = worst_u = 0.0
    for d in range(32):
        dk, du = synth.fd_direction(d, n * n, n * n, seed=8)
        dkd, dud = dk.reshape(n, n), du.reshape(n, n)
        fd = (loss_at(kap + eps_k * dkd, u0) - loss_at(kap - eps_k * dkd, u0)) / (2 * eps_k)
        an = float(np.dot(gk_h.ravel(), dk))
        ek = abs(fd - an) / max(abs(an), 1e-3 * nk)
        assert ek <= 1e-6, (d, fd, an)
        fd = (loss_at(kap, u0 + eps_u * dud) - loss_at(kap, u0 - eps_u * dud)) / (2 * eps_u)
        an = float(np.dot(gu_h.ravel(), du))
        eu = abs(fd - an) / max(abs(an), ngu)
        assert eu <= 1e-9, (d, fd, an)
        worst_k, worst_u = max(worst_k, ek), max(worst_u, eu)
    print("32 directions: worst relative FD error kappa %.2e, u0 %.2e" % (worst_k, worst_u))
    assert L0 > 0


@pytest.mark.parametrize("steps,every", [(100, 10), (500, 23)])
def test_adjoint_full_size_vs_oracle(dev, steps, every):
    """The full 2048^2 field of the differentiation workload (same kappa_ref,
    kappa and u0) over 100 steps checkpointed every 10, and over the
    workload's own 500 steps checkpointed every 23 (the oracle then stores
    all 501 states, 16 GB, and takes about 90 s): loss, dL/dkappa and dL/du0
    element by element against the oracle's reverse accumulation, norm-wise
    relative 1e-11 (measured 2.5e-14 and 3.5e-13 at 500 steps)."""
    n, c = 2048, 0.15
    kref, kap, u0, _ = synth.adjoint_input(n)
    tgt = oracle.varcoef2d(u0, kref, c, steps)
    oloss, ogk, ogu = oracle.varcoef2d_adjoint(u0, kap, tgt, c, steps)
    bu0, bk, bt = up(dev, u0), up(dev, kap), up(dev, tgt)
    uT, lam, loss_b = dev.buffer(u0.nbytes), dev.buffer(u0.nbytes), dev.buffer(8)
    hxc.varcoef_forward_run(dev, bu0, bk, n, n, c, steps, uT)[0].get()
    hxc.sqerr_seed(dev, uT, bt, lam, loss_b, n * n).get()
    # the oracle adds the 2048^2 squares one after the other: relative error
    # bound n 2^-53 = 4.7e-10 (the GPU's fixed-order tree is far tighter)
    assert abs(down(loss_b, 1)[0] - oloss) <= 4.7e-10 * oloss
    for mode in ("fused", "plain"):
        gk, gu, _, _ = adjoint(dev, u0, kap, down(lam, u0.shape), c, steps, every, mode)
        assert rel(gk, ogk) <= TOLG, mode
        assert rel(gu, ogu) <= TOLG, mode


def test_autograd_function(dev):
    torch = pytest.importorskip("torch")
    from paper_1810_11482_b300.autograd import VarcoefHeat
    n, steps, c = 64, 30, 0.15
    kref, kap, _, _ = synth.adjoint_input(n)
    u0 = synth.bumps2d(n, n, seed=7, nbumps=4, sigma=0.1)
    tgt = oracle.varcoef2d(u0, kref, c, steps)
    tu = torch.tensor(u0, device="cuda", requires_grad=True)
    tk = torch.tensor(kap, device="cuda", requires_grad=True)
    tt = torch.tensor(tgt, device="cuda")
    uT = VarcoefHeat.apply(tu, tk, c, steps, 0)
    loss = ((uT - tt) ** 2).sum()
    loss.backward()
    oloss, ogk, ogu = oracle.varcoef2d_adjoint(u0, kap, tgt, c, steps)
    assert abs(loss.item() - oloss) <= 1e-12 * oloss
    assert rel(tk.grad.cpu().numpy(), ogk) <= TOLG
    assert rel(tu.grad.cpu().numpy(), ogu) <= TOLG
