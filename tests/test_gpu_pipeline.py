"""The whole pass (initial state, integration, correlation integral,
bootstrap statistics) as one Pipeline: eager, captured in a CUDA graph and
replayed, and as separate public calls all give bit-identical outputs; the
counts equal the oracle's on the same fields.  Two parameter groups (FHN and
GM on 32x32) exercise the persistent batched launch."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_14742_b300 as pk
    return pk


def make(p):
    gds = [W.group(W.FHN, 32, 32, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, 300, (-0.05, 0.05), 501, 3),
           W.group(W.GM, 32, 32, (2.5e-4, 0.01, 1.0, 0.5), 2 ** -8, 200, (0.0, 0.01), 502, 1)]
    groups = [p.Group.from_dict(g) for g in gds]
    sets = [(16, 16, g["species_mask"]) for g in gds]
    return gds, p.Pipeline(groups, sets, M=8, b=1.3, T=50, seed=77)


def snapshot(pipe):
    out = {"fields": pipe.sim.fields.clone(), "residual": pipe.residual.clone(), "bins": pipe.bins.clone(),
           "C": pipe.C.clone()}
    for i, o in enumerate(pipe.cil_out):
        out["counts%d" % i] = o["counts"].clone()
        out["radii%d" % i] = o["radii"].clone()
    for k, v in pipe.stats.items():
        out["stats_" + k] = v.clone()
    return out


def test_pipeline_eager_graph_and_separate_calls_agree(p):
    gds, pipe = make(p)
    pipe.run()
    torch.cuda.synchronize()
    eager = snapshot(pipe)
    for o in pipe.cil_out:
        assert int(o["n_rechecked"]) >= 0
    pipe.capture()
    for _ in range(2):
        pipe.replay()
        torch.cuda.synchronize()
        again = snapshot(pipe)
        for k in eager:
            assert torch.equal(eager[k], again[k]), k

    # the same pass as separate public calls
    _, pipe2 = make(p)
    pipe2.sim.reinit()
    pipe2.sim.integrate()
    for i, (X1, X2) in enumerate(pipe2.views):
        c = p.cil(X1, X2, b=1.3, M=8)
        assert torch.equal(c["bins"], eager["bins"][i])
        assert torch.equal(c["counts"], eager["counts%d" % i])
    torch.cuda.synchronize()
    assert torch.equal(pipe2.sim.fields, eager["fields"])

    # counts against the oracle on the same FP32 fields
    for i, g in enumerate(gds):
        f = pipe.sim.group_fields(i).cpu().numpy()
        X = oracle.patterns(f, g["species_mask"])
        o = oracle.cil(X[:16], X[16:32], b=1.3, M=8)
        assert np.array_equal(eager["bins"][i].cpu().numpy(), o["bins"])
        assert np.array_equal(eager["counts%d" % i].cpu().numpy(), o["counts"])


def test_rdode_pipeline_with_rkc_and_linear_law(p):
    # the RD-ODE likelihood pass of Table 1 (64 nodes, t in [0, 50], linear
    # radii, M = 13) plus a 2-D group on the adaptive integrator: eager and
    # graph replay bit-identical, counts equal the oracle's on the same fields
    gds = [W.group(W.RDODE, 64, 40, W.RDODE_THETA0, 50.0 / 1024, 1024, (0.0, 2.0), 601, 3),
           W.group(W.FHN, 32, 40, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -8, 512, (-0.05, 0.05), 602, 1)]
    groups = [p.Group.from_dict(g) for g in gds]
    sets = [(20, 20, g["species_mask"]) for g in gds]
    pipe = p.Pipeline(groups, sets, M=13, b=None, T=50, seed=78, integrator="rkc",
                      rkc=dict(rtol=1e-5, atol=1e-5), law="linear")
    pipe.run()
    torch.cuda.synchronize()
    eager = snapshot(pipe)
    st = pipe.rkc_stats.cpu().numpy()
    assert (st[:, 0] > 0).all()
    pipe.capture()
    pipe.replay()
    torch.cuda.synchronize()
    rep = snapshot(pipe)
    for k in eager:
        a, b = eager[k], rep[k]
        if a.dtype == torch.float64:        # bit patterns (a non-PD group's scalars are NaN)
            a, b = a.view(torch.int64), b.view(torch.int64)
        assert torch.equal(a, b), k
    for i, (X1, X2) in enumerate(pipe.views):
        o = oracle.cil(X1.cpu().numpy(), X2.cpu().numpy(), M=13, law="linear")
        assert np.array_equal(pipe.cil_out[i]["counts"].cpu().numpy(), o["counts"])
        assert np.array_equal(pipe.bins[i].cpu().numpy(), o["bins"])


def test_pipeline_with_the_semi_implicit_stepper(p):
    # a likelihood pass on the semi-implicit stepper (FHN 64 and GM 32 at
    # steps far above the explicit diffusive limit): eager and graph replay
    # bit-identical, fields within tolerance of the oracle's semi-implicit
    # run, counts equal the oracle's on the same fields
    from oracle import imex as OI
    gds = [W.group(W.FHN, 64, 24, (2.9e-4, 0.048, 9.7, 0.93), 2 ** -5, 120, (-0.05, 0.05), 611, 1),
           W.group(W.GM, 32, 24, (2.5e-4, 0.01, 1.0, 0.48), 2 ** -4, 100, (0.0, 0.01), 612, 3)]
    groups = [p.Group.from_dict(g) for g in gds]
    sets = [(12, 12, g["species_mask"]) for g in gds]
    pipe = p.Pipeline(groups, sets, M=10, b=1.3, T=40, seed=79, integrator="imex")
    pipe.sim.reinit()
    w0 = [pipe.sim.group_fields(i)[:2].cpu().numpy().copy() for i in range(2)]
    pipe.run()
    torch.cuda.synchronize()
    eager = snapshot(pipe)
    for i, g in enumerate(groups):
        want = OI.imex_run(g.model, g.params, g.dt, g.n_steps, w0[i])
        got = pipe.sim.group_fields(i)[:2].cpu().numpy().astype(np.float64)
        err = (np.abs(got - want).reshape(2, 2, -1).max(-1) / np.abs(want).reshape(2, 2, -1).max(-1)).max()
        assert err <= 1e-5, (i, err)
    pipe.capture()
    pipe.replay()
    torch.cuda.synchronize()
    rep = snapshot(pipe)
    for k in eager:
        a, b = eager[k], rep[k]
        if a.dtype == torch.float64:
            a, b = a.view(torch.int64), b.view(torch.int64)
        assert torch.equal(a, b), k
    for i, (X1, X2) in enumerate(pipe.views):
        o = oracle.cil(X1.cpu().numpy(), X2.cpu().numpy(), 1.3, 10)
        assert np.array_equal(pipe.cil_out[i]["counts"].cpu().numpy(), o["counts"])


@pytest.mark.parametrize("kind", ["rkc", "imex"])
def test_first_call_of_a_handle_captures_in_a_graph(p, kind):
    """The stabilised RK2 and semi-implicit step tables belong to the
    handle (formed by rd_init on its device), so the very first
    rd_integrate_rkc / rd_integrate_imex call of a fresh handle launches
    only the integrator (no table set-up, no allocation, no synchronise)
    and can be captured in a CUDA graph; replaying it gives the eager
    result bit for bit."""
    import ctypes
    g = p.Group(W.FHN, 64, 4, (2.8e-4, 0.05, 10.0, 0.95), 2 ** -10, 120, (-0.05, 0.05), 77)
    sim = p.Simulation([g])
    sz = ctypes.c_size_t()
    assert p.lib().rd_tables_size(sim._arr, 1, ctypes.byref(sz)) == 0
    assert sim.table_bytes() == sz.value > 0

    def call(s):
        if kind == "rkc":
            s.integrate_rkc(h0=2 ** -10, s_fixed=6, n_fixed=40, stats=False)
        else:
            s.integrate_imex()

    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    n0 = p.lib().rd_kernel_launches()
    with torch.cuda.graph(graph):
        call(sim)
    assert p.lib().rd_kernel_launches() - n0 == 1
    graph.replay()
    torch.cuda.synchronize()
    eager = p.Simulation([g])
    call(eager)
    torch.cuda.synchronize()
    assert torch.equal(sim.fields, eager.fields)
    assert sim.sync_status() == 0 and eager.sync_status() == 0


def test_concurrent_correlation_integrals_match_sequential(p):
    """Twelve groups: their correlation integrals forked over four side
    streams (each with its own workspace) give the same bits as one after
    another on the calling stream, eagerly and replayed from a graph."""
    gds = [W.group(W.FHN if i % 2 == 0 else W.GM, 32, 32,
                   (2.8e-4, 0.05, 10.0, 0.95) if i % 2 == 0 else (2.5e-4, 0.01, 1.0, 0.5),
                   2 ** -8, 60 + 10 * i, (-0.05, 0.05) if i % 2 == 0 else (0.0, 0.01), 900 + i, 1 + 2 * (i % 2))
           for i in range(12)]
    outs = []
    for ns in (1, 4):
        groups = [p.Group.from_dict(g) for g in gds]
        pipe = p.Pipeline(groups, [(16, 16, g["species_mask"]) for g in gds], M=8, b=1.3, T=40, seed=5,
                          cil_streams=ns)
        assert len(pipe.side) == (0 if ns == 1 else ns)
        pipe.run()
        torch.cuda.synchronize()
        outs.append(snapshot(pipe))
        if ns > 1:
            pipe.capture()
            pipe.replay()
            torch.cuda.synchronize()
            again = snapshot(pipe)
            for k in outs[-1]:
                assert torch.equal(outs[-1][k], again[k]), k
    for k in outs[0]:
        assert torch.equal(outs[0][k], outs[1][k]), k


def rel_field_err(a, b):
    a = np.asarray(a, np.float64).reshape(2, -1)
    b = np.asarray(b, np.float64).reshape(2, -1)
    return float((np.abs(a - b).max(-1) / np.abs(b).max(-1)).max())


def test_c4_full_size_in_the_benchmark_launch(p):
    """The benchmark's step, c4 in full: 64 parameter vectors x 128
    realisations, FHN and GM at 64^2 (10^4 steps) and 128^2 (2 x 10^4) in
    one persistent launch, the 64 correlation integrals forked over side
    streams and the batched bootstrap statistics, as bench.py times it.
    Sampled against the oracle for the first group of every model and grid:
    the last realisation's fields at the full horizon (field tolerance
    1e-5), the correlation integral's radii, bins and counts on the GPU's
    fields, and the bootstrap counts, mean, covariance and factor (bit for
    bit)."""
    cfg = W.config("c4")
    gds = cfg["groups"]
    n1, n2, M, b, T = cfg["n1"], cfg["n2"], cfg["M"], cfg["b"], cfg["T_res"]
    groups = [p.Group.from_dict(g) for g in gds]
    pipe = p.Pipeline(groups, [(n1, n2, g["species_mask"]) for g in gds], M, b, T, cfg["seed"])
    assert len(pipe.side) > 1
    picks = {}
    for i, g in enumerate(gds):
        picks.setdefault((g["model"], g["G"]), i)
    assert len(picks) == 4
    f0 = {i: pipe.sim.group_fields(i)[-1:].cpu().numpy().astype(np.float64) for i in picks.values()}
    pipe.run(reinit=False)
    torch.cuda.synchronize()
    assert pipe.sim.sync_status() == 0
    for i in picks.values():
        g = gds[i]
        ref = oracle.step(g["model"], g["params"], g["dt"], g["n_steps"], f0[i])
        assert rel_field_err(pipe.sim.group_fields(i)[-1:].cpu().numpy(), ref) <= 1e-5, i
        X = oracle.patterns(pipe.sim.group_fields(i).cpu().numpy(), g["species_mask"])
        o = oracle.cil(X[:n1], X[n1:n1 + n2], b=b, M=M)
        assert float(pipe.cil_out[i]["radii"][0]) == o["R0"]
        assert np.array_equal(pipe.cil_out[i]["radii"][1:].cpu().numpy(), o["radii"])
        assert np.array_equal(pipe.bins[i].cpu().numpy(), o["bins"])
        assert np.array_equal(pipe.cil_out[i]["counts"].cpu().numpy(), o["counts"])
        so = oracle.synlik(o["bins"], M, T, cfg["seed"] + i, y_obs=o["counts"] / float(n1 * n2))
        assert np.array_equal(pipe.stats["Y"][i].cpu().numpy(), so["Y"])
        assert np.array_equal(pipe.stats["mu"][i].cpu().numpy(), so["mu"])
        assert np.array_equal(pipe.stats["cov"][i].cpu().numpy(), so["cov"])
        assert int(pipe.stats["status"][i]) == so["status"]
        if so["status"] == 0:
            assert np.array_equal(pipe.stats["chol"][i].cpu().numpy(), so["chol"])
