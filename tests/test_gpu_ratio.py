"""Fused quasi-simultaneous ratio (blip_eval_ratio) against the FP64 oracle.

For each walker, D[j][l] = psi_l(r_j) is built by the oracle at the current
configuration and inverted in FP64; every electron then gets a Gaussian trial
move r'_j, and the GPU returns sum_l {psi, grad psi, lap psi}_l(r'_j)
(D^{-1})_{lj}.  Checks:
  * against the oracle's outputs contracted in FP64, under the propagated
    per-output bound plus the FP32 summation of the dot product;
  * the matrix-determinant lemma: the value component equals
    det(D with row j replaced by psi(r'_j)) / det(D);
  * with no move (r'_j = r_j) the ratio is 1 (D D^{-1} = I);
  * the optional new-row output equals blip_eval's values bitwise.
"""
import numpy as np
import pytest

import blip_inputs as bi
import oracle
import pins

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TAU32 = 8e-6


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1204_1121_gb300 as pb
    return pb


def _setup(n_orb=96, walkers=3, seed=5):
    grid = (14, 12, 16)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, n_orb, seed=seed, sigma=2.0)
    rng = np.random.default_rng(seed)
    cur = [rng.uniform(0, 1, size=(n_orb, 3)) @ lat for _ in range(walkers)]
    Dinv = []
    for w in range(walkers):
        v, _, _ = oracle.eval_stencil(grid, lat, tab, cur[w])
        Dinv.append(np.linalg.inv(v))
    return grid, lat, tab, cur, Dinv


@pytest.mark.parametrize("storage,sort", [("f32", 0), ("f32", 1), ("bf16", 0)])
def test_ratio_matches_oracle_and_determinant_lemma(pb, storage, sort):
    grid, lat, tab, cur, Dinv = _setup()
    n = tab.shape[-1]
    rng = np.random.default_rng(17)
    new = [c + rng.normal(0, 0.3, size=c.shape) for c in cur]
    pos = np.concatenate(new)
    offs = np.arange(0, len(pos) + 1, n, dtype=np.int32)
    # electron j of walker w uses column j of that walker's inverse
    cols = np.ascontiguousarray(np.concatenate([Di.T for Di in Dinv]), dtype=np.float32)  # [E][n]
    kind = pb.F32 if storage == "f32" else pb.BF16
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    dpos = torch.from_numpy(pos).cuda()
    ratio, vals = t.eval_ratio(dpos, torch.from_numpy(cols).cuda(),
                               torch.from_numpy(offs).cuda(), with_values=True, sort=sort)
    torch.cuda.synchronize()
    ratio = ratio.cpu().numpy().astype(np.float64)
    rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    c64 = cols.astype(np.float64)
    ref = np.stack([(rv * c64).sum(1), (rg[:, 0] * c64).sum(1), (rg[:, 1] * c64).sum(1),
                    (rg[:, 2] * c64).sum(1), (rl * c64).sum(1)], 1)
    tau = TAU32 + (2.0 ** -8 if storage == "bf16" else 0.0)
    outs = [rv, rg[:, 0], rg[:, 1], rg[:, 2], rl]
    for k in range(5):
        mk = mag[:, 0] if k == 0 else (mag[:, k] if k < 4 else mag[:, 4])
        bound = (np.abs(c64) * tau * mk).sum(1) \
            + 2 * (n / 32 + 8) * 2.0 ** -24 * (np.abs(outs[k] * c64)).sum(1) + 1e-12
        assert (np.abs(ratio[:, k] - ref[:, k]) <= bound).all(), k
    # matrix-determinant lemma on the value ratio, all in FP64: the new row
    # dotted with column j of the FP64 inverse equals det(D_j') / det(D); the
    # GPU value ratio then differs from it by the bound above plus the FP32
    # rounding of the column (2^-24 sum |psi c|)
    for w in range(len(cur)):
        D, _, _ = oracle.eval_stencil(grid, lat, tab, cur[w])
        d0 = np.linalg.slogdet(D)
        newv, _, _ = oracle.eval_stencil(grid, lat, tab, new[w])
        for j in (0, n // 2, n - 1):
            Dj = D.copy()
            Dj[j] = newv[j]
            s1, l1 = np.linalg.slogdet(Dj)
            lemma = s1 * d0[0] * np.exp(l1 - d0[1])
            dot64 = float(newv[j] @ Dinv[w][:, j])
            assert abs(dot64 - lemma) <= 1e-9 * (1 + abs(lemma)) * np.linalg.cond(D)
            e = w * n + j
            slack = 2.0 ** -24 * float(np.abs(newv[j] * Dinv[w][:, j]).sum())
            assert abs(ratio[e, 0] - lemma) <= (np.abs(c64[e]) * tau * mag[e, 0]).sum() \
                + 2 * (n / 32 + 8) * 2.0 ** -24 * float(np.abs(rv[e] * c64[e]).sum()) + slack + 1e-12
    if storage == "f32":
        ev, _, _ = t.eval(dpos)
        assert np.array_equal(ev.cpu().numpy(), vals.cpu().numpy())
    assert t.status() == 0


def test_ratio_is_one_without_a_move(pb):
    grid, lat, tab, cur, Dinv = _setup(n_orb=64, walkers=2, seed=8)
    n = tab.shape[-1]
    pos = np.concatenate(cur)
    cols = np.ascontiguousarray(np.concatenate([Di.T for Di in Dinv]), dtype=np.float32)
    t = pb.BlipTable(grid, lat, tab)
    ratio, _ = t.eval_ratio(torch.from_numpy(pos).cuda(), torch.from_numpy(cols).cuda())
    r = ratio.cpu().numpy().astype(np.float64)[:, 0]
    rv, _, _, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    c64 = cols.astype(np.float64)
    # sum_l psi_l (D^{-1})_{lj} = 1; the FP32 column adds 2^-24 sum |psi c|, the
    # GPU adds its per-output bound and the FP32 dot-product summation
    s_abs = (np.abs(rv * c64)).sum(1)
    bound = (np.abs(c64) * TAU32 * mag[:, 0]).sum(1) + (2 * (n / 32 + 8) + 1) * 2.0 ** -24 * s_abs
    assert (np.abs(r - 1.0) <= bound + 1e-12).all()


def test_ratio_rejects_complex_tables_and_bad_args(pb):
    grid = (6, 6, 6)
    tab = bi.smooth_random_table(grid, 4, seed=1, is_complex=True)
    t = pb.BlipTable(grid, np.eye(3) * 6, tab, storage=pb.C64)
    pos = torch.zeros((3, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(pb.BlipError):
        t.eval_ratio(pos, torch.zeros((3, 8), dtype=torch.float32, device="cuda"))
    L = pb.lib()
    assert L.blip_eval_ratio(None, None, 1, None, 0, None, None, None, 0, None) == -1


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_ratio_precision_tio2_shape(pb, storage):
    """The acceptance ratio on the TiO2-shaped table (768 orbitals, two
    walkers of 1,536 electrons, two spins of 768), the GPU use of the
    paper's single-precision orbitals (Sec. V.B): every electron's trial
    move r'_j = r_j + N(0, 0.3^2) is judged by xi_j = sum_l psi_l(r'_j)
    (D_sigma^{-1})_{lj} (Eq. 11.12.23.1).  Checked against the FP64 ratio of
    the oracle's orbitals under the propagated bound (coefficient rounding u
    for quantised tables, FP32 rounding, the FP32 column), and every
    Metropolis decision min(1, xi^2) > U (U seeded uniforms) that the GPU
    ratio flips must lie inside that bound's band.  Prints the relative
    error and the number of flipped decisions."""
    import json
    w = bi.workload("tio2")
    tab = w.table()
    base, offs = bi.walker_positions(w.lattice, 2, 1536, 1536, seed=103, move_sigma=0.0)
    moved, _ = bi.walker_positions(w.lattice, 2, 1536, 1536, seed=103)
    n = 768
    cols = np.empty((len(moved), n), dtype=np.float32)
    for wk in range(2):
        v, _, _ = oracle.eval_stencil(w.grid, w.lattice, tab, base[1536 * wk:1536 * (wk + 1)])
        for sp in range(2):
            j0 = 1536 * wk + n * sp
            Dinv = np.linalg.inv(v[n * sp:n * (sp + 1), :n])
            cols[j0:j0 + n] = Dinv.T                   # electron j: column j of D^{-1}
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16}[storage]
    # the ratio contracts the first n orbitals: a table of exactly those
    t = pb.BlipTable(w.grid, w.lattice, tab[..., :n], storage=kind)
    ratio, _ = t.eval_ratio(torch.from_numpy(moved).cuda(), torch.from_numpy(cols).cuda(),
                            torch.from_numpy(offs).cuda(), sort=1)
    torch.cuda.synchronize()
    xi = ratio.cpu().numpy().astype(np.float64)[:, 0]
    rv, _, _, mag = oracle.eval_stencil(w.grid, w.lattice, tab[..., :n], moved, absmag=True)
    c64 = cols.astype(np.float64)
    ref = (rv * c64).sum(1)
    tau = TAU32 + {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[storage]
    bound = (np.abs(c64) * tau * mag[:, 0]).sum(1) \
        + 2 * (n / 32 + 8) * 2.0 ** -24 * np.abs(rv * c64).sum(1)
    if kind == pb.F16:                                 # FP16 subnormal floor
        s_l = np.abs(tab[..., :n]).reshape(-1, n).max(0)
        bound += 2.0 ** -25 * (np.abs(c64) * s_l[None, :]).sum(1)
    err = np.abs(xi - ref)
    assert (err <= bound).all(), float(np.max(err / bound))
    U = bi.uniform(bi.stream_key(103, 0xACC), np.arange(len(moved), dtype=np.uint64))
    acc_ref = np.minimum(1.0, ref ** 2) > U
    acc_gpu = np.minimum(1.0, xi ** 2) > U
    flips = acc_ref != acc_gpu
    band = np.abs(np.minimum(1.0, ref ** 2) - U) <= 2 * np.abs(ref) * bound + bound ** 2
    assert (band[flips]).all()
    rel = err / np.abs(ref)
    print("\n" + json.dumps({"storage": storage, "max_rel_err": float(rel.max()),
                             "rms_rel_err": float(np.sqrt(np.mean(rel ** 2))),
                             "median_rel_err": float(np.median(rel)),
                             "flipped_decisions": int(flips.sum()), "moves": len(moved),
                             "accepted_ref": int(acc_ref.sum())}))
    assert t.status() == 0


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_ratio_tensor_cores_dense_batch(pb, storage):
    """A dense batch (about 3 electrons per cell, crowded cells, a NaN
    position) in cell order goes to the tensor-core ratio: the contraction of
    the matrix-product outputs with each electron's column, reduced on the
    chip in a fixed order.  Checked against the FP64 oracle's contraction
    under the tensor-core per-output bound (1.6e-5 sum_s |W_o(s)| |a_ls|, the
    coefficient rounding of 16-bit storage, the FP16 subnormal floor) carried
    through the column, plus the FP32 summation; the new-row output equals
    the tensor-core evaluation's values bitwise; the CUDA-core sorted path
    (sort = 2) meets its own bound on the same batch; repeated runs agree
    bitwise."""
    grid = (12, 10, 14)
    lat = pins.triclinic_lattice()
    n = 300                                          # 3 M tiles, the last ragged
    tab = bi.smooth_random_table(grid, n, seed=61, sigma=2.0)
    rng = np.random.default_rng(62)
    ncell = int(np.prod(grid))
    u = rng.uniform(0, 1, size=(3 * ncell, 3))
    crowd = [(np.array(c) + rng.uniform(0.05, 0.95, size=(k, 3))) / np.array(grid)
             for c, k in (((1, 2, 3), 60), ((5, 0, 11), 26), ((0, 9, 13), 25))]
    u = np.concatenate([u] + crowd)
    u[:40] += rng.integers(-5, 6, size=(40, 3))
    pos = np.concatenate([u @ lat, [[np.nan, 1.0, 2.0]]])
    pos = pos[rng.permutation(len(pos))]
    E = len(pos)
    offs = np.array([0, 1000, 1000, 3100, E], dtype=np.int32)
    cols = rng.normal(0.0, 1.0, size=(E, n)).astype(np.float32)
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16}[storage]
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    dpos = torch.from_numpy(pos).cuda()
    dcols = torch.from_numpy(cols).cuda()
    doffs = torch.from_numpy(offs).cuda()
    ratio, vals = t.eval_ratio(dpos, dcols, doffs, with_values=True, sort=1)
    again, _ = t.eval_ratio(dpos, dcols, doffs, with_values=True, sort=1)
    core, _ = t.eval_ratio(dpos, dcols, doffs, sort=2)
    t.set_kernel(12, 1, 1, 1)
    ev, _, _ = t.eval(dpos, doffs)
    torch.cuda.synchronize()
    bad = np.isnan(pos).any(1)
    r = ratio.cpu().numpy().astype(np.float64)
    assert np.isnan(r[bad]).all() and np.isnan(vals.cpu().numpy()[bad]).all()
    assert torch.equal(torch.nan_to_num(ratio, nan=3.0), torch.nan_to_num(again, nan=3.0))
    assert torch.equal(torch.nan_to_num(vals, nan=3.0), torch.nan_to_num(ev, nan=3.0))
    ok = ~bad
    rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos[ok], absmag=True)
    c64 = cols[ok].astype(np.float64)
    outs = [rv, rg[:, 0], rg[:, 1], rg[:, 2], rl]
    u_q = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[storage]
    floor = np.zeros((ok.sum(), 5, n))
    if storage in ("f32", "f16"):
        s_l = (2.0 if storage == "f32" else 1.0) * np.abs(tab.reshape(-1, n)).max(0)
        ones = np.ones(tuple(grid) + (1,))
        _, _, _, sw = oracle.eval_stencil(grid, lat, ones, pos[ok], absmag=True)
        floor = 2.0 ** -25 * (64.0 + sw[:, :, 0])[:, :, None] * s_l[None, None, :]
    worst = 0.0
    for k in range(5):
        ref = (outs[k] * c64).sum(1)
        summ = 2 * (n / 32 + 8) * 2.0 ** -24 * np.abs(outs[k] * c64).sum(1)
        tc_b = (np.abs(c64) * ((1.6e-5 + u_q) * mag[:, k] + floor[:, k])).sum(1) + summ + 1e-30
        core_f = floor[:, k] if storage == "f16" else 0.0
        core_b = (np.abs(c64) * ((TAU32 + u_q) * mag[:, k] + core_f)).sum(1) + summ + 1e-30
        e_tc = np.abs(r[ok, k] - ref) / tc_b
        worst = max(worst, float(e_tc.max()))
        assert (e_tc <= 1.0).all(), (k, float(e_tc.max()))
        e_core = np.abs(core.cpu().numpy().astype(np.float64)[ok, k] - ref)
        assert (e_core <= core_b).all(), k
    print(f"\nstorage {storage}: worst tensor-core ratio error / bound {worst:.3g}")
    assert t.status() == pb.STATUS_NONFINITE_POS


@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_ratio_tensor_core_operand_kernel(pb, storage):
    """Without the new-row output, a dense batch in cell order goes to the
    ratio kernel that contracts the orbitals on the tensor cores first,
    Y[k][j] = sum_l a[k][l] c_j[l] over the part's 128 union rows k, then
    sum_k W_o^(j)[k] Y[k][j] in the epilogue.  Its bound: the tensor-core
    coefficient bound (1.6e-5 C_o, storage rounding, FP16 subnormal floor)
    carried through the column; the FP32 accumulation over the 16 L/128
    K steps and the 64-term reduction, (16 L/128 + 16) 2^-24 sum_l |c_l|
    C_o(l); the 16-bit split of c'_l = c_l s_l / sigma (FP16: 2^-22 relative
    plus 2^-25 sigma absolute, sigma the power of two at or above
    max_l |c_l s_l|; BF16: 2^-17 relative), carried through |psi_l|; and the
    FP32 summation term of the other tests.  Repeated runs agree bitwise;
    with the new-row output requested the evaluation kernel's ratio epilogue
    runs instead and also meets its bound."""
    grid = (12, 10, 14)
    lat = pins.triclinic_lattice()
    n = 300
    tab = bi.smooth_random_table(grid, n, seed=63, sigma=2.0)
    rng = np.random.default_rng(64)
    ncell = int(np.prod(grid))
    u = rng.uniform(0, 1, size=(3 * ncell, 3))
    crowd = [(np.array(c) + rng.uniform(0.05, 0.95, size=(k, 3))) / np.array(grid)
             for c, k in (((2, 3, 4), 40), ((7, 1, 0), 26), ((11, 9, 13), 25))]
    u = np.concatenate([u] + crowd)
    u[:40] += rng.integers(-5, 6, size=(40, 3))
    pos = np.concatenate([u @ lat, [[1.0, np.inf, 2.0]]])
    pos = pos[rng.permutation(len(pos))]
    E = len(pos)
    # columns of mixed magnitude per electron (the per-electron scale sigma)
    cols = (rng.normal(0.0, 1.0, size=(E, n)) *
            10.0 ** rng.uniform(-3, 3, size=(E, 1))).astype(np.float32)
    kind = {"f32": pb.F32, "bf16": pb.BF16, "f16": pb.F16}[storage]
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    dpos = torch.from_numpy(pos).cuda()
    dcols = torch.from_numpy(cols).cuda()
    r1, _ = t.eval_ratio(dpos, dcols, sort=1)
    r2, _ = t.eval_ratio(dpos, dcols, sort=1)
    rv_, _ = t.eval_ratio(dpos, dcols, with_values=True, sort=1)
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(r1, nan=3.0), torch.nan_to_num(r2, nan=3.0))
    bad = ~np.isfinite(pos).all(1)
    r = r1.cpu().numpy().astype(np.float64)
    assert np.isnan(r[bad]).all()
    ok = ~bad
    rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos[ok], absmag=True)
    c64 = cols[ok].astype(np.float64)
    outs = [rv, rg[:, 0], rg[:, 1], rg[:, 2], rl]
    u_q = {"f32": 0.0, "bf16": 2.0 ** -8, "f16": 2.0 ** -11}[storage]
    amax = np.abs(tab.reshape(-1, n)).max(0)
    s_l = 2.0 ** np.ceil(np.log2(amax)) if storage == "f32" else amax
    floor = np.zeros((ok.sum(), 5, n))
    if storage in ("f32", "f16"):
        ones = np.ones(tuple(grid) + (1,))
        _, _, _, sw = oracle.eval_stencil(grid, lat, ones, pos[ok], absmag=True)
        floor = 2.0 ** -25 * (64.0 + sw[:, :, 0])[:, :, None] * \
            ((2.0 if storage == "f32" else 1.0) * amax)[None, None, :]
    sig = 2.0 ** np.ceil(np.log2(np.abs(c64 * s_l[None, :]).max(1)))
    mt = (n + 127) // 128
    worst = 0.0
    rw = rv_.cpu().numpy().astype(np.float64)
    for k in range(5):
        ref = (outs[k] * c64).sum(1)
        summ = 2 * (n / 32 + 8) * 2.0 ** -24 * np.abs(outs[k] * c64).sum(1)
        base = (np.abs(c64) * ((1.6e-5 + u_q) * mag[:, k] + floor[:, k])).sum(1)
        acc = (16 * mt + 16) * 2.0 ** -24 * (np.abs(c64) * mag[:, k]).sum(1)
        if storage == "bf16":
            split = 2.0 ** -17 * (np.abs(outs[k]) * np.abs(c64)).sum(1)
        else:
            split = (np.abs(outs[k]) * (2.0 ** -22 * np.abs(c64) +
                                        2.0 ** -25 * sig[:, None] / s_l[None, :])).sum(1)
        bound = base + acc + split + summ + 1e-30
        e = np.abs(r[ok, k] - ref) / bound
        worst = max(worst, float(e.max()))
        assert (e <= 1.0).all(), (k, float(e.max()))
        # the evaluation kernel's ratio epilogue (new rows requested)
        eb = (np.abs(c64) * ((1.6e-5 + u_q) * mag[:, k] + floor[:, k])).sum(1) + summ + 1e-30
        assert (np.abs(rw[ok, k] - ref) <= eb).all(), k
    print(f"\nstorage {storage}: worst operand-kernel ratio error / bound {worst:.3g}")
    assert t.status() == pb.STATUS_NONFINITE_POS


@pytest.mark.parametrize("storage,n,misalign", [("f32", 130, False), ("bf16", 300, True)])
def test_ratio_operand_kernel_scalar_paths(pb, storage, n, misalign):
    """The ratio kernel's paths without 16-byte column loads: an orbital
    count that is not a multiple of 4 (130: a ragged second orbital tile),
    and columns whose base address is 4 bytes off 16-byte alignment.  Both
    against the FP64 oracle under the operand kernel's bound."""
    grid = (10, 9, 12)
    lat = pins.triclinic_lattice()
    tab = bi.smooth_random_table(grid, n, seed=65, sigma=2.0)
    rng = np.random.default_rng(66)
    pos = rng.uniform(0, 1, size=(3 * int(np.prod(grid)), 3)) @ lat
    E = len(pos)
    cols = (rng.normal(0.0, 1.0, size=(E, n)) *
            10.0 ** rng.uniform(-2, 2, size=(E, 1))).astype(np.float32)
    kind = pb.F32 if storage == "f32" else pb.BF16
    t = pb.BlipTable(grid, lat, tab, storage=kind)
    if misalign:
        buf = torch.empty(E * n + 1, dtype=torch.float32, device="cuda")
        dcols = buf[1:].view(E, n)
        dcols.copy_(torch.from_numpy(cols))
        assert dcols.data_ptr() % 16 != 0
    else:
        dcols = torch.from_numpy(cols).cuda()
    r, _ = t.eval_ratio(torch.from_numpy(pos).cuda(), dcols, sort=1)
    torch.cuda.synchronize()
    r = r.cpu().numpy().astype(np.float64)
    rv, rg, rl, mag = oracle.eval_stencil(grid, lat, tab, pos, absmag=True)
    c64 = cols.astype(np.float64)
    outs = [rv, rg[:, 0], rg[:, 1], rg[:, 2], rl]
    u_q = {"f32": 0.0, "bf16": 2.0 ** -8}[storage]
    amax = np.abs(tab.reshape(-1, n)).max(0)
    s_l = 2.0 ** np.ceil(np.log2(amax)) if storage == "f32" else amax
    floor = np.zeros((E, 5, n))
    if storage == "f32":
        ones = np.ones(tuple(grid) + (1,))
        _, _, _, sw = oracle.eval_stencil(grid, lat, ones, pos, absmag=True)
        floor = 2.0 ** -25 * (64.0 + sw[:, :, 0])[:, :, None] * (2.0 * amax)[None, None, :]
    sig = 2.0 ** np.ceil(np.log2(np.abs(c64 * s_l[None, :]).max(1)))
    mt = (n + 127) // 128
    for k in range(5):
        ref = (outs[k] * c64).sum(1)
        summ = 2 * (n / 32 + 8) * 2.0 ** -24 * np.abs(outs[k] * c64).sum(1)
        base = (np.abs(c64) * ((1.6e-5 + u_q) * mag[:, k] + floor[:, k])).sum(1)
        acc = (16 * mt + 16) * 2.0 ** -24 * (np.abs(c64) * mag[:, k]).sum(1)
        if storage == "bf16":
            split = 2.0 ** -17 * (np.abs(outs[k]) * np.abs(c64)).sum(1)
        else:
            split = (np.abs(outs[k]) * (2.0 ** -22 * np.abs(c64) +
                                        2.0 ** -25 * sig[:, None] / s_l[None, :])).sum(1)
        bound = base + acc + split + summ + 1e-30
        assert (np.abs(r[:, k] - ref) <= bound).all(), (k, float((np.abs(r[:, k] - ref) / bound).max()))
    assert t.status() == 0


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_ratio_tensor_cores_full_precision_batch(pb, storage):
    """The fused ratio at full size, in the launch configuration bench.py
    times (1,024 walkers x 1,536 trial moves on the TiO2-shaped table, cell
    order, no new rows: the operand kernel), with seeded N(0,1) columns made
    on the device: 48 sampled electrons against the FP64 oracle's
    contraction under the operand kernel's bound."""
    w = bi.workload("tio2")
    tab = w.table()
    wp = bi.workload("tio2_precision")
    pos, offs = wp.positions()
    E, n = len(pos), tab.shape[-1]
    kind = pb.F32 if storage == "f32" else pb.BF16
    t = pb.BlipTable(w.grid, w.lattice, tab, storage=kind)
    g = torch.Generator(device="cuda")
    g.manual_seed(67)
    dcols = torch.randn((E, n), generator=g, device="cuda", dtype=torch.float32)
    r, _ = t.eval_ratio(torch.from_numpy(pos).cuda(), dcols, torch.from_numpy(offs).cuda(), sort=1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(68)
    idx = np.unique(np.concatenate([[0, E - 1], rng.integers(0, E, 46)]))
    got = r[idx].cpu().numpy().astype(np.float64)
    c64 = dcols[idx].cpu().numpy().astype(np.float64)
    del dcols
    rv, rg, rl, mag = oracle.eval_stencil(w.grid, w.lattice, tab, pos[idx], absmag=True)
    outs = [rv, rg[:, 0], rg[:, 1], rg[:, 2], rl]
    u_q = {"f32": 0.0, "bf16": 2.0 ** -8}[storage]
    amax = np.abs(tab.reshape(-1, n)).max(0)
    s_l = 2.0 ** np.ceil(np.log2(amax)) if storage == "f32" else amax
    floor = np.zeros((len(idx), 5, n))
    if storage == "f32":
        ones = np.ones(tuple(w.grid) + (1,))
        _, _, _, sw = oracle.eval_stencil(w.grid, w.lattice, ones, pos[idx], absmag=True)
        floor = 2.0 ** -25 * (64.0 + sw[:, :, 0])[:, :, None] * (2.0 * amax)[None, None, :]
    sig = 2.0 ** np.ceil(np.log2(np.abs(c64 * s_l[None, :]).max(1)))
    mt = (n + 127) // 128
    worst = 0.0
    for k in range(5):
        ref = (outs[k] * c64).sum(1)
        summ = 2 * (n / 32 + 8) * 2.0 ** -24 * np.abs(outs[k] * c64).sum(1)
        base = (np.abs(c64) * ((1.6e-5 + u_q) * mag[:, k] + floor[:, k])).sum(1)
        acc = (16 * mt + 16) * 2.0 ** -24 * (np.abs(c64) * mag[:, k]).sum(1)
        if storage == "bf16":
            split = 2.0 ** -17 * (np.abs(outs[k]) * np.abs(c64)).sum(1)
        else:
            split = (np.abs(outs[k]) * (2.0 ** -22 * np.abs(c64) +
                                        2.0 ** -25 * sig[:, None] / s_l[None, :])).sum(1)
        bound = base + acc + split + summ + 1e-30
        e = np.abs(got[:, k] - ref) / bound
        worst = max(worst, float(e.max()))
        assert (e <= 1.0).all(), (k, float(e.max()))
    print(f"\nstorage {storage}: full-size ratio, worst error / bound {worst:.3g}")
    assert t.status() == 0
