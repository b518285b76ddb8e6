"""Serving (emsurf_submit / emsurf_poll): requests of uneven lattice size and
right-hand-side count run concurrently on one GPU; each result equals the
result of the same request solved alone; admission refuses requests that can
never fit; polling reports pending and unknown tickets."""
import numpy as np
import pytest

from paper_1911_04576_gb300 import workloads as W

pytestmark = pytest.mark.gpu

A, H = W.PERIOD, W.BOX_H


def _requests(B):
    rng = np.random.default_rng(42)
    specs = [(2, 2, 2, 1), (3, 3, 2, 2), (4, 3, 3, 1), (2, 5, 2, 3), (3, 2, 3, 2)]
    out = []
    for nx, ny, n, R in specs:
        T = 3
        sides = rng.uniform(0.15, 0.45, T) * W.LAMBDA
        sides[0] = 0.0                                        # one empty type
        tmap = rng.integers(0, T, nx * ny)
        waves = [W.plane_waves(W.Workload("w", 1, 1, 1, 1, 0, 0, angles=[(th, ph, "theta")]))[0]
                 for th, ph in zip(rng.uniform(0, 50, R), rng.uniform(0, 360, R))]
        kh = np.array([w_[0] for w_ in waves])
        eh = np.array([w_[1] for w_ in waves])
        _, _, nu = B.emsurf_setup_overlap(n, nx, ny)
        out.append(dict(a=A, b=A, h=H, n=n, nx=nx, ny=ny, k0=W.K0, patch_sides=sides,
                        patch_z=W.PATCH_Z, patch_n=3, type_map=tmap, khat=kh, ehat=eh,
                        precision=B.MIXED, rtol=1e-9, restart=30, max_iters=6000, nu=nu, R=R))
    return out


def _run(B, reqs, max_active):
    sv = B.emsurf_server_create(0, 0, max_active)
    xs, tickets = [], []
    for r in reqs:
        x = np.zeros((r["R"], r["nu"]), np.complex128)
        kw = {k: v for k, v in r.items() if k not in ("nu", "R")}
        q, keep = B.make_request(x_out=x, **kw)
        tickets.append(B.emsurf_submit(sv, q, keep))
        xs.append(x)
    res = [B.emsurf_wait(sv, t, 600000) for t in tickets]
    sv.close()
    return xs, res


def test_each_result_same_alone_and_in_the_mix(emsurf_lib):
    from paper_1911_04576_gb300 import binding as B
    reqs = _requests(B)
    xs_mix, res_mix = _run(B, reqs, 3)
    for r in res_mix:
        assert r["status"] == B.EMSURF_OK and r["info"]["converged"] == 1
        assert r["info"]["rel_residual"] <= 1e-9
    for i, r in enumerate(reqs):
        xa, ra = _run(B, [r], 1)
        assert np.linalg.norm(xa[0] - xs_mix[i]) <= 1e-12 * np.linalg.norm(xa[0])


def test_admission_and_polling(emsurf_lib):
    from paper_1911_04576_gb300 import binding as B
    r = _requests(B)[0]
    kw = {k: v for k, v in r.items() if k not in ("nu", "R")}
    q, keep = B.make_request(**kw)
    need = B.emsurf_request_bytes(q)
    # a budget below one request's estimate: refused at submit
    sv = B.emsurf_server_create(0, need // 2, 2)
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_submit(sv, q, keep)
    assert e.value.status == B.EMSURF_EBUSY
    sv.close()
    # a budget that fits one request at a time: both still complete
    sv = B.emsurf_server_create(0, int(need * 1.5), 2)
    t1 = B.emsurf_submit(sv, q, keep)
    t2 = B.emsurf_submit(sv, q, keep)
    first = B.emsurf_poll(sv, t1)                   # normally still pending
    r1 = first if first is not None else B.emsurf_wait(sv, t1, 600000)
    r2 = B.emsurf_wait(sv, t2, 600000)
    assert r1["status"] == B.EMSURF_OK and r2["status"] == B.EMSURF_OK
    with pytest.raises(B.EmsurfError) as e:
        B.emsurf_poll(sv, t1)                       # collected already
    assert e.value.status == B.EMSURF_EINVAL
    sv.close()


def test_resident_blocks_are_reused(emsurf_lib):
    """Requests of one lattice with other type maps and rhs counts read the
    Fourier-domain blocks and the library macromodels the first one left
    resident (cache hits), and give the result of a server that builds
    everything per request; a request that needs another spectrum form (one
    rhs: half of the FP32 spectrum) gets an entry of its own."""
    from paper_1911_04576_gb300 import binding as B
    rng = np.random.default_rng(7)
    n, nx, ny, T = 2, 4, 3, 3
    sides = rng.uniform(0.15, 0.45, T) * W.LAMBDA
    _, _, nu = B.emsurf_setup_overlap(n, nx, ny)
    reqs = []
    for R in (2, 3, 2, 1):
        waves = [W.plane_waves(W.Workload("w", 1, 1, 1, 1, 0, 0, angles=[(th, 0.0, "theta")]))[0]
                 for th in rng.uniform(0, 50, R)]
        reqs.append(dict(a=A, b=A, h=H, n=n, nx=nx, ny=ny, k0=W.K0, patch_sides=sides, patch_z=W.PATCH_Z,
                         patch_n=3, type_map=rng.integers(0, T, nx * ny), khat=np.array([w_[0] for w_ in waves]),
                         ehat=np.array([w_[1] for w_ in waves]), precision=B.MIXED, rtol=1e-9, restart=30,
                         max_iters=6000, precond_overlap=0.6 * A / n, slab_t=W.SLAB_T, slab_eps=W.EPS_SLAB,
                         ring_layers=2, nu=nu, R=R))

    def serve(cache):
        sv = B.emsurf_server_create(0, 0, 1, cache=cache)
        xs, res = [], []
        for r in reqs:                       # one at a time: the first builds, the rest read
            x = np.zeros((r["R"], r["nu"]), np.complex128)
            q, keep = B.make_request(x_out=x, **{k: v for k, v in r.items() if k not in ("nu", "R")})
            res.append(B.emsurf_wait(sv, B.emsurf_submit(sv, q, keep), 600000))
            xs.append(x)
        stats = B.emsurf_server_stats(sv)
        sv.close()
        return xs, res, stats

    xc, rc, stats = serve(True)
    xn, rn, _ = serve(False)
    assert [r["cache_hit"] for r in rc] == [0, 1, 1, 0]
    assert [r["cache_hit"] for r in rn] == [0, 0, 0, 0]
    assert stats[1] == 2 and stats[2] == 1 and stats[0] > 0       # two lattice forms, one library
    for a, b, r in zip(xc, xn, rc):
        assert r["status"] == B.EMSURF_OK and r["info"]["rel_residual"] <= 1e-9
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_cancel_withdraws_only_queued_requests(emsurf_lib):
    """One worker: the first request runs, the later ones wait; withdrawing a
    queued one gives ECANCELED, a request that already ran is not withdrawn."""
    from paper_1911_04576_gb300 import binding as B
    reqs = _requests(B)
    sv = B.emsurf_server_create(0, 0, 1)
    tickets, keeps = [], []
    for r in reqs[:3]:
        kw = {k: v for k, v in r.items() if k not in ("nu", "R")}
        q, keep = B.make_request(**kw)
        tickets.append(B.emsurf_submit(sv, q, keep))
        keeps.append(keep)
    withdrawn = B.emsurf_cancel(sv, tickets[2])
    r0 = B.emsurf_wait(sv, tickets[0], 600000)
    assert r0["status"] == B.EMSURF_OK
    r2 = B.emsurf_wait(sv, tickets[2], 600000)
    assert r2["status"] == (B.EMSURF_ECANCELED if withdrawn else B.EMSURF_OK)
    r1 = B.emsurf_wait(sv, tickets[1], 600000)
    assert r1["status"] == B.EMSURF_OK
    with pytest.raises(B.EmsurfError):
        B.emsurf_cancel(sv, 987654321)
    sv.close()


def test_solve_wall_time_limit(emsurf_lib):
    """max_ms stops the solve at the first restart past it: ENOTCONV with the
    best iterate, long before the iteration budget."""
    import torch
    from paper_1911_04576_gb300 import binding as B
    w = W.WORKLOADS["lattice16x16_k576"]
    idx, sgn, nu = B.emsurf_setup_overlap(w.n, w.nx, w.ny)
    zl = B.emsurf_setup_slab_zlevels(H, w.n, W.SLAB_T)
    L = torch.empty((2 * w.ny - 1, 2 * w.nx - 1, w.E, w.E), dtype=torch.complex128, device="cuda")
    K = torch.empty_like(L)
    B.emsurf_tabulate_offsets(A, A, H, w.n, w.nx, w.ny, W.K0, L, K, zlevels=zl)
    Z = torch.empty((w.n_types, w.K, w.K), dtype=torch.complex128, device="cuda")
    B.emsurf_macromodel_slab_patch(A, A, H, w.n, zl, W.patch_sides(w), w.patch_n, W.RING_LAYERS,
                                   W.EPS_SLAB, W.K0, Z)
    coef = (1j * W.K0, 1.0, -1.0, 1j * W.K0)
    h = B.emsurf_create(w.nx, w.ny, w.E, nu, W.type_map(w), Z, L, K, coef, idx, sgn, precision=B.FP64,
                        tables_on_device=True)
    V = torch.empty((1, nu), dtype=torch.complex128, device="cuda")
    waves = W.plane_waves(w)
    B.emsurf_excitation(h, A, A, H, w.n, W.K0, [waves[0][0]], [waves[0][1]], V, zlevels=zl)
    X = torch.zeros_like(V)
    # unpreconditioned FP64 GMRES needs ~1800 iterations here
    st, info = B.emsurf_solve(h, V, X, rtol=1e-6, restart=30, max_iters=20000, solver=B.SOLVER_FP64,
                              max_ms=1.0)
    assert st == B.EMSURF_ENOTCONV
    assert info[0]["iters"] <= 60 and info[0]["rel_residual"] > 1e-6
    assert np.isfinite(X.cpu().numpy()).all()
    with pytest.raises(B.EmsurfError):
        B.emsurf_solve(h, V, X, rtol=1e-6, max_ms=-1.0)
    h.close()


def test_admission_keeps_the_library_it_reuses(emsurf_lib):
    """A second lattice of the same cell library under a budget of one
    request's estimate: if room has to be made, it is made by evicting the
    first lattice's operator, never the library the new request was
    admitted to reuse (evicting it would leave the request waiting for an
    entry nobody builds); the request completes within the wait limit."""
    from paper_1911_04576_gb300 import binding as B
    rng = np.random.default_rng(11)
    n, T = 2, 3
    sides = rng.uniform(0.15, 0.45, T) * W.LAMBDA
    reqs = []
    for nx in (4, 5):
        waves = [W.plane_waves(W.Workload("w", 1, 1, 1, 1, 0, 0, angles=[(20.0, 0.0, "theta")]))[0]]
        reqs.append(dict(a=A, b=A, h=H, n=n, nx=nx, ny=nx, k0=W.K0, patch_sides=sides, patch_z=W.PATCH_Z,
                         patch_n=3, type_map=rng.integers(0, T, nx * nx), khat=np.array([w_[0] for w_ in waves]),
                         ehat=np.array([w_[1] for w_ in waves]), precision=B.MIXED, rtol=1e-8, restart=30,
                         max_iters=6000, slab_t=W.SLAB_T, slab_eps=W.EPS_SLAB, ring_layers=2))
    qs = [B.make_request(**r) for r in reqs]
    need = max(B.emsurf_request_bytes(q) for q, _ in qs)
    # room for one request's build: the second forces an eviction
    sv = B.emsurf_server_create(0, need + (1 << 20), 1, cache=True)
    res = []
    for q, keep in qs:
        t = B.emsurf_submit(sv, q, keep)
        res.append(B.emsurf_wait(sv, t, 300000))      # ETIMEDOUT (raised) if it waits for ever
    stats = B.emsurf_server_stats(sv)
    sv.close()
    assert all(r["status"] == B.EMSURF_OK for r in res)
    assert stats[2] == 1                             # the shared library stayed resident
