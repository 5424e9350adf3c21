"""Batched instances (csrc/batch.cu): one persistent operator launch over many uneven
meshes, lock-step GMRES with a captured restart cycle, and the autotuner.

The batched operator evaluates every element and node sum in the same order as the
single-mesh launch (only the assignment of tiles to CTAs differs); the two kernels are
separate instantiations of one body, so the compiler may contract a different set of
multiply-adds: results agree to a few ulps, not bit for bit.  Batched GMRES follows
the same algorithm per instance (flexible GMRES with each instance's network as well); its solutions are checked against the residual of
the per-instance operator and against per-instance solves (two solutions that both
meet rel-res 1e-10 differ by up to the condition number times 1e-10: measured up to
2.2e-5 on these NS blocks, so the solutions are compared at 1e-4)."""
import numpy as np
import pytest

from tests.gpu_helpers import DEV, T
from tests.helpers import desc_small

pytestmark = pytest.mark.gpu

import torch  # noqa: E402

from paper_2402_10348_gb300 import fsi  # noqa: E402
from workloads import cavity, random_state  # noqa: E402


def _instances(sizes, seed=0):
    descs = [cavity(n).desc for n in sizes] + [desc_small(n=(7, 11, 5)), desc_small(n=(9, 4, 13))]
    stream = torch.cuda.Stream()
    meshes, states = [], []
    for k, d in enumerate(descs):
        m = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(m, stream)
        meshes.append(m)
        states.append(tuple(T(a) for a in random_state(d, seed + k, amp_v=0.3)))
    torch.cuda.synchronize()
    return descs, meshes, states, stream


def _concat(parts):
    return torch.cat([p.reshape(-1) for p in parts]).contiguous()


@pytest.mark.parametrize("flags", [fsi.FSI_ELASTIC_AUG, fsi.FSI_ELASTIC_AUG | fsi.FSI_FP32])
@pytest.mark.parametrize("block", [fsi.FSI_BLOCK_NS, fsi.FSI_BLOCK_AC(1), fsi.FSI_BLOCK_B(0)])
def test_batched_jvp_matches_per_instance(flags, block):
    descs, meshes, states, stream = _instances([8, 12, 16, 10])
    b = fsi.fsi_batch_create(meshes, block=block, m=30)
    rng = np.random.default_rng(5)
    dxs = [T(rng.normal(size=b.offsets[i + 1] - b.offsets[i])) for i in range(b.n)]
    ys = []
    with torch.cuda.stream(stream):
        if block == fsi.FSI_BLOCK_AC(1):
            for m in meshes:
                fsi.fsi_set_ac_coeffs(m, 1, 0.37, 0.11)
        for i, m in enumerate(meshes):
            y = torch.zeros_like(dxs[i])
            fsi.fsi_jvp(m, block, *states[i], dxs[i], y, flags)
            ys.append(y)
        yb = torch.zeros(b.offsets[-1], dtype=torch.float64, device=DEV)
        launches0 = b.layout()[2]
        fsi.fsi_batch_jvp(b, states, _concat(dxs), yb, flags)
        launches1 = b.layout()[2]
    torch.cuda.synchronize()
    ref = _concat(ys)
    err = float((yb - ref).abs().max() / ref.abs().max())
    print(f"block {block} flags {flags}: max relative difference {err:.2e}")
    assert err <= (1e-6 if flags & fsi.FSI_FP32 else 1e-13)
    # one operator launch (+ the float copy); the float32 NS product from per-instance
    # coefficients is an element launch and a node launch
    assert launches1 - launches0 <= (3 if block == fsi.FSI_BLOCK_NS and flags & fsi.FSI_FP32 else 2)


@pytest.mark.parametrize("precision", [fsi.FSI_PREC_FP64, fsi.FSI_PREC_FP32_IR])
def test_batched_gmres_matches_per_instance_solves(precision):
    descs, meshes, states, stream = _instances([8, 12, 16], seed=3)
    b = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=30)
    rhs = []
    with torch.cuda.stream(stream):
        for i, m in enumerate(meshes):
            r = torch.zeros(b.offsets[i + 1] - b.offsets[i], dtype=torch.float64, device=DEV)
            fsi.fsi_residual(m, fsi.FSI_BLOCK_NS, *states[i], r)
            rhs.append(r)
    torch.cuda.synchronize()
    o = fsi.solve_opts(m=30, rtol=1e-10, max_iter=4000, precision=precision, ir_inner_rtol=1e-3, ir_max=60)
    sols = []
    with torch.cuda.stream(stream):
        for i, m in enumerate(meshes):
            x = torch.zeros_like(rhs[i])
            fsi.fsi_gmres(m, fsi.FSI_BLOCK_NS, *states[i], rhs[i], x, o)
            sols.append(x)
        xb = torch.zeros(b.offsets[-1], dtype=torch.float64, device=DEV)
        infos = fsi.fsi_batch_gmres(b, states, _concat(rhs), xb, o)
        # the same solve without the captured graph: identical kernels, identical result
        fsi.fsi_batch_set_graph(b, False)
        xb2 = torch.zeros_like(xb)
        fsi.fsi_batch_gmres(b, states, _concat(rhs), xb2, o)
    torch.cuda.synchronize()
    assert torch.equal(xb, xb2)
    for i, m in enumerate(meshes):
        xi = xb[b.offsets[i]:b.offsets[i + 1]]
        assert infos[i].rel_res <= 1e-10
        t = torch.zeros_like(xi)
        with torch.cuda.stream(stream):
            fsi.fsi_jvp(m, fsi.FSI_BLOCK_NS, *states[i], xi.contiguous(), t)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(rhs[i] - t) / torch.linalg.norm(rhs[i])) <= 1.5e-10
        assert float(torch.linalg.norm(xi - sols[i]) / torch.linalg.norm(sols[i])) <= 1e-4


def test_autotuner_picks_a_shape_and_caches_it(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("FSI_AUTOTUNE_CACHE", str(cache))
    descs, meshes, states, stream = _instances([8, 12, 16, 20])
    b = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=30)
    with torch.cuda.stream(stream):
        tm, gm, us = fsi.fsi_batch_autotune(b, states)
    torch.cuda.synchronize()
    assert tm in (1, 2, 4, 8) and gm in (1, 2, 4) and us > 0.0
    assert b.layout()[:2] == (tm, gm)
    line = cache.read_text().strip().splitlines()[-1].split()
    assert (int(line[1]), int(line[2])) == (tm, gm)
    b2 = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=30)  # the cache is read at creation
    assert b2.layout()[:2] == (tm, gm)


def test_batched_products_and_solves_against_the_oracle():
    """Each instance of a batch of uneven meshes against the oracle: the batched NS, AC
    and B products (float64, 1e-10 of max) and the batched float64 NS solve (rel-res
    1e-12) against the oracle's exact solve of the same system (sparse LU of the probed
    Jacobian): residual with the oracle's operator <= 1e-11, solution within 1e-6."""
    from oracle import blocks
    from oracle.assemble import assemble, direct_solve
    from oracle.fields import Problem, State
    descs, meshes, states, stream = _instances([5, 7], seed=9)
    host = [tuple(a.cpu().numpy() for a in st) for st in states]
    coeffs = {"gamma": {1: 0.37}, "beta": {1: 0.11}}
    for block, name in ((fsi.FSI_BLOCK_NS, "ns"), (fsi.FSI_BLOCK_AC(1), ("ac", 1)), (fsi.FSI_BLOCK_B(0), ("b", 0))):
        b = fsi.fsi_batch_create(meshes, block=block, m=30)
        rng = np.random.default_rng(7)
        dxs = [rng.normal(size=b.offsets[i + 1] - b.offsets[i]) for i in range(b.n)]
        yb = torch.zeros(b.offsets[-1], dtype=torch.float64, device=DEV)
        with torch.cuda.stream(stream):
            for m in meshes:
                fsi.fsi_set_ac_coeffs(m, 1, 0.37, 0.11)
            fsi.fsi_batch_jvp(b, states, T(np.concatenate(dxs)), yb, fsi.FSI_ELASTIC_AUG)
        torch.cuda.synchronize()
        for i, d in enumerate(descs):
            pb, st = Problem(d), State(*host[i])
            ref = blocks.jvp(pb, st, name, dxs[i], coeffs)
            got = yb[b.offsets[i]:b.offsets[i + 1]].cpu().numpy()
            assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max(), (name, i)
    b = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=30)
    rhs = [-blocks.residual(Problem(d), State(*host[i]), "ns") for i, d in enumerate(descs)]
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=8000)
    xb = torch.zeros(b.offsets[-1], dtype=torch.float64, device=DEV)
    with torch.cuda.stream(stream):
        infos = fsi.fsi_batch_gmres(b, states, T(np.concatenate(rhs)), xb, o)
    torch.cuda.synchronize()
    for i, d in enumerate(descs):
        pb, st = Problem(d), State(*host[i])
        A = assemble(pb, st, "ns")
        exact = direct_solve(A, rhs[i])
        got = xb[b.offsets[i]:b.offsets[i + 1]].cpu().numpy()
        assert infos[i].rel_res <= 1e-12
        assert np.linalg.norm(rhs[i] - blocks.jvp(pb, st, "ns", got)) <= 1e-11 * np.linalg.norm(rhs[i])
        assert np.linalg.norm(got - exact) <= 1e-6 * np.linalg.norm(exact), i


def _cavity_states(sizes):
    from oracle.gridcell import apply_rules, signed_distance_phi
    descs, xs = [], []
    for n in sizes:
        wl = cavity(n)
        d = wl.desc
        phi, _ = signed_distance_phi(d, wl.surfaces[0], d.eps, wl.grid_cells)
        x = np.zeros((d.ncomp, d.nn))
        x[4:4 + d.n_phase] = apply_rules(d, {0: phi}, wl.rules, d.eps)
        x[4 + d.n_phase: 4 + d.n_phase + 3] = 1.0
        descs.append(d)
        xs.append(x)
    return descs, xs


@pytest.mark.parametrize("precision", [fsi.FSI_PREC_FP64, fsi.FSI_PREC_FP32_IR])
def test_batched_time_steps_match_per_instance_steps_and_the_oracle(precision):
    """Three uneven cavities advanced by batched partitioned steps (one batched solve per
    block kind and nonlinear iteration; the Allen-Cahn blocks of both phases of every
    instance in one batch) against per-instance fsi_step, two steps of three fixed
    nonlinear iterations, every solve to rel-res 1e-12: the fields agree to 1e-9
    (float64) and 1e-6 (float32 refinement).  The 5^3 instance is also held to the
    oracle's steps with exact block solves (1e-10 in float64)."""
    from oracle import step as ostep
    from oracle.fields import Problem, State
    descs, xs = _cavity_states([5, 7, 6])
    stream = torch.cuda.Stream()
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=6000, precision=precision, ir_inner_rtol=1e-3, ir_max=60)
    singles, batched, meshes_b = [], [], []
    for d, x in zip(descs, xs):
        ms = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(ms, stream)
        mb = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(mb, stream)
        singles.append((ms, [T(x), T(x), T(np.zeros_like(x))]))
        batched.append([T(x), T(x), T(np.zeros_like(x))])
        meshes_b.append(mb)
    stepper = fsi.fsi_batch_stepper_create(meshes_b, m=30)
    ref = State(xs[0].copy(), xs[0].copy(), np.zeros_like(xs[0]))
    for s in range(2):
        with torch.cuda.stream(stream):
            for ms, st in singles:
                fsi.fsi_step(ms, *st, k_max=3, fixed_iters=True, solve=o)
            infos = fsi.fsi_batch_step(stepper, batched, k_max=3, fixed_iters=True, solve=o)
        torch.cuda.synchronize()
        ostep.time_step(Problem(descs[0]), ref, ostep.StepOptions(k_max=3, fixed_nl_iters=True, direct=True))
        for i, d in enumerate(descs):
            assert infos[i].nl_iters == 3
            a = batched[i][1].cpu().numpy().reshape(d.ncomp, d.nn)
            b = singles[i][1][1].cpu().numpy().reshape(d.ncomp, d.nn)
            for sl in (slice(0, 3), slice(3, 4), slice(4, 6), slice(6, 12)):
                e = np.linalg.norm(a[sl] - b[sl]) / np.linalg.norm(b[sl])
                assert e <= (1e-9 if precision == fsi.FSI_PREC_FP64 else 1e-6), (s, i, sl, e)
                if i == 0 and precision == fsi.FSI_PREC_FP64:
                    eo = np.linalg.norm(a[sl] - ref.xn[sl]) / np.linalg.norm(ref.xn[sl])
                    assert eo <= 1e-10, (s, sl, eo)


@pytest.mark.parametrize("precision", [fsi.FSI_PREC_FP64, fsi.FSI_PREC_FP32_IR])
def test_batched_flexible_gmres_with_the_network(precision):
    """Flexible GMRES over a batch with each instance's own network (untrained seeded
    weights, network and Jacobi directions alternately): every instance reaches rel-res
    1e-10, checked with its own float64 operator, and its solution agrees with the
    per-instance float64 Jacobi solve at 5e-4 (both meet 1e-10, so they differ by up to the
    condition number times 2e-10: measured 1.1e-4 with the float32 basis of the batched
    refinement's inner solves).  Without FSI_PC_ALTERNATE the solve still returns (network directions
    only); an AC batch refuses the network."""
    from workloads import he_normal_weights
    descs, meshes, states, stream = _instances([8, 12, 16], seed=3)
    pcs = []
    for m in meshes:
        pc = fsi.fsi_pc_create(m)
        fsi.fsi_pc_set_weights(pc, he_normal_weights(pc.fan, 7))
        fsi.fsi_set_pc(m, pc)
        pcs.append(pc)
    b = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_NS, m=30)
    rhs = []
    with torch.cuda.stream(stream):
        for i, m in enumerate(meshes):
            r = torch.zeros(b.offsets[i + 1] - b.offsets[i], dtype=torch.float64, device=DEV)
            fsi.fsi_residual(m, fsi.FSI_BLOCK_NS, *states[i], r)
            rhs.append(r)
    torch.cuda.synchronize()
    o = fsi.solve_opts(m=30, rtol=1e-10, max_iter=4000, precision=precision, ir_inner_rtol=1e-3, ir_max=60)
    o64 = fsi.solve_opts(m=30, rtol=1e-10, max_iter=4000)
    jac = []
    with torch.cuda.stream(stream):
        for i, m in enumerate(meshes):
            x = torch.zeros_like(rhs[i])
            fsi.fsi_gmres(m, fsi.FSI_BLOCK_NS, *states[i], rhs[i], x, o64)  # reference: float64 Jacobi
            jac.append(x)
        ol = fsi.fsi_solve_opts.from_buffer_copy(o)
        ol.precond = fsi.FSI_PC_LEARNED
        ol.flags |= fsi.FSI_PC_ALTERNATE
        xb = torch.zeros(b.offsets[-1], dtype=torch.float64, device=DEV)
        infos = fsi.fsi_batch_gmres(b, states, _concat(rhs), xb, ol)
    torch.cuda.synchronize()
    for i, m in enumerate(meshes):
        xi = xb[b.offsets[i]:b.offsets[i + 1]].contiguous()
        assert infos[i].rel_res <= 1e-10
        t = torch.zeros_like(xi)
        with torch.cuda.stream(stream):
            fsi.fsi_jvp(m, fsi.FSI_BLOCK_NS, *states[i], xi, t)
        torch.cuda.synchronize()
        assert float(torch.linalg.norm(rhs[i] - t) / torch.linalg.norm(rhs[i])) <= 1.5e-10
        assert float(torch.linalg.norm(xi - jac[i]) / torch.linalg.norm(jac[i])) <= 5e-4
    # network directions only: the call completes (convergence is not asserted)
    ol.flags &= ~fsi.FSI_PC_ALTERNATE
    ol.max_iter = 120
    with torch.cuda.stream(stream):
        fsi.fsi_batch_gmres(b, states, _concat(rhs), xb, ol, allow_noconv=True)
    torch.cuda.synchronize()
    ba = fsi.fsi_batch_create(meshes, block=fsi.FSI_BLOCK_AC(0), m=30)
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_batch_gmres(ba, states, torch.zeros(ba.offsets[-1], dtype=torch.float64, device=DEV),
                            torch.zeros(ba.offsets[-1], dtype=torch.float64, device=DEV), ol)
    assert e.value.code == fsi.FSI_EINVAL


def test_batched_time_steps_with_the_network():
    """Batched steps whose NS solves use flexible GMRES with each instance's network
    (alternate directions; Jacobi for the Allen-Cahn and B blocks) against per-instance
    Jacobi steps: two steps of three fixed nonlinear iterations, every solve to rel-res
    1e-12 (solves may stop on a stall near that floor, as in the Jacobi steps), the fields
    agree to 1e-8."""
    from workloads import he_normal_weights
    descs, xs = _cavity_states([5, 7, 6])
    stream = torch.cuda.Stream()
    o = fsi.solve_opts(m=30, rtol=1e-12, max_iter=6000)
    singles, batched, meshes_b, pcs = [], [], [], []
    for d, x in zip(descs, xs):
        ms = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(ms, stream)
        mb = fsi.fsi_create_mesh(d)
        fsi.fsi_set_stream(mb, stream)
        pc = fsi.fsi_pc_create(mb)
        fsi.fsi_pc_set_weights(pc, he_normal_weights(pc.fan, 5))
        fsi.fsi_set_pc(mb, pc)
        pcs.append(pc)
        singles.append((ms, [T(x), T(x), T(np.zeros_like(x))]))
        batched.append([T(x), T(x), T(np.zeros_like(x))])
        meshes_b.append(mb)
    stepper = fsi.fsi_batch_stepper_create(meshes_b, m=30)
    ol = fsi.fsi_solve_opts.from_buffer_copy(o)
    ol.precond = fsi.FSI_PC_LEARNED
    ol.flags |= fsi.FSI_PC_ALTERNATE
    for s in range(2):
        with torch.cuda.stream(stream):
            for ms, st in singles:
                fsi.fsi_step(ms, *st, k_max=3, fixed_iters=True, solve=o)
            infos = fsi.fsi_batch_step(stepper, batched, k_max=3, fixed_iters=True, solve=ol)
        torch.cuda.synchronize()
        for i, d in enumerate(descs):
            assert infos[i].nl_iters == 3
            a = batched[i][1].cpu().numpy().reshape(d.ncomp, d.nn)
            b = singles[i][1][1].cpu().numpy().reshape(d.ncomp, d.nn)
            for sl in (slice(0, 3), slice(3, 4), slice(4, 6), slice(6, 12)):
                e = np.linalg.norm(a[sl] - b[sl]) / np.linalg.norm(b[sl])
                assert e <= 1e-8, (s, i, sl, e)
