"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: relative Frobenius error per trial vector <= 1e-11 for the FP64
path and <= 1e-5 for the FP32 path (errors of FP32 pair products, FFTs and
accumulation over ~10^2-10^3 pairs stay near 1e-6).
"""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu

TOL = {T.PREC_FP64: 1e-11, T.PREC_FP32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def _workload(n, a, ecut, nocc, nb, seed=0, sf=False, nocc_tgt=None):
    npw = T.sphere_size(n, a, ecut)
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=npw, nocc_src=nocc, nb=nb, seed=seed, spin_flip=sf,
                               nocc_tgt=nocc_tgt)


def _rel_err(got, want):
    got = got.reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _run(torch, wl, prec, mask=T.TERMS_ALL, X=None, tiling=None):
    sys_ = T.system_from_workload(wl, precision=prec, term_mask=mask)
    if isinstance(tiling, dict):
        sys_.set_tuning(**tiling)
    elif tiling:
        sys_.set_tuning(*tiling)
    X = wl.X if X is None else X
    Xd = torch.from_numpy(X).to("cuda", sys_.complex_dtype)
    out = sys_.apply(Xd)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.complex128)
    sys_.close()
    return res


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_tiny_full_operator(torch, prec):
    """24^3 grid, 8 orbitals, 4 trial vectors: the plain FP64 spin-conserving case."""
    wl = _workload(24, 10.0, 10.0, 8, 4)
    want = O.system_from_workload(wl).apply(wl.X)
    got = _run(torch, wl, prec)
    assert _rel_err(got, want).max() < TOL[prec]


@pytest.mark.parametrize("term", [T.TERM_D_KIN, T.TERM_D_VLOC, T.TERM_D_EXX, T.TERM_K1E_H, T.TERM_K1E_XC,
                                  T.TERM_K1D, T.TERM_D_EXX | T.TERM_PROJ, T.TERM_K1D | T.TERM_PROJ])
def test_each_term_fp64(torch, term):
    wl = _workload(12, 7.0, 4.0, 4, 3, seed=3)
    want = O.system_from_workload(wl).apply(wl.X, term)
    got = _run(torch, wl, T.PREC_FP64, mask=term)
    assert _rel_err(got, want).max() < 1e-11


@pytest.mark.parametrize("n,a,ecut,nocc,nb", [(8, 6.0, 3.2, 3, 2), (12, 7.0, 4.0, 3, 1), (16, 8.0, 6.0, 5, 2),
                                               (24, 10.0, 10.0, 3, 1), (32, 9.0, 12.0, 6, 2),
                                               (36, 9.0, 14.0, 5, 1), (48, 10.0, 20.0, 4, 1),
                                               (64, 11.0, 25.0, 3, 1), (72, 13.48, 25.0, 3, 1),
                                               (80, 15.0, 25.0, 2, 1), (96, 17.97, 25.0, 2, 1),
                                               (108, 20.2, 25.0, 2, 1), (128, 23.96, 25.0, 1, 1)])
def test_every_grid_plan(torch, n, a, ecut, nocc, nb):
    """One system per supported radix plan (8, 4x3, 16, 8x3, 8x4, 4x9, 16x3, 8x8, 8x9,
    16x5, 12x8, 12x9, 8x16; 128^3 in FP32 only)."""
    wl = _workload(n, a, ecut, nocc, nb, seed=n)
    want = O.system_from_workload(wl).apply(wl.X)
    for prec in (T.PREC_FP64, T.PREC_FP32):
        if n == 128 and prec == T.PREC_FP64:
            continue  # the FP64 128^3 plane does not fit in shared memory
        got = _run(torch, wl, prec)
        assert _rel_err(got, want).max() < TOL[prec], (n, prec)
        # the pair convolutions on the n grid itself too, where a smaller exchange grid exists
        s = T.system_from_workload(wl, precision=prec)
        nx = s.query()["n_exchange"]
        s.close()
        assert nx == EXCHANGE_GRID.get(n, n), (n, nx)
        if nx != n:
            got = _run(torch, wl, prec, tiling=dict(exchange_grid=0))
            assert _rel_err(got, want).max() < TOL[prec], (n, prec, "n grid")


# smallest supported N_x < n with N_x > 4 max|m_i| for the cells of test_every_grid_plan
EXCHANGE_GRID = {36: 32, 72: 64, 80: 72, 108: 96, 128: 108}


def test_exchange_grid_is_the_same_operator(torch):
    """72^3 cell at 25 Ha (max |m_i| = 15): the pair-convolution terms on 64^3 against the same terms
    on 72^3 and the oracle (on 72^3), for the Tamm-Dancoff operator, the Z-vector operator (K2 terms),
    K1d alone with stored tau, and with the compressed exchange inside D."""
    wl = _workload(72, 13.48, 25.0, 6, 2, seed=19)
    S = O.system_from_workload(wl)
    for prec in (T.PREC_FP64, T.PREC_FP32):
        tight = 1e-12 if prec == T.PREC_FP64 else 2e-6
        s = T.system_from_workload(wl, precision=prec)
        assert s.query()["n_exchange"] == 64
        Xd = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)

        def both(mask):
            s.set_terms(mask)
            s.set_tuning(exchange_grid=1)
            small = s.apply(Xd).cpu().numpy().astype(np.complex128)
            s.set_tuning(exchange_grid=0)
            assert s.query()["n_exchange"] == 72
            full = s.apply(Xd).cpu().numpy().astype(np.complex128)
            s.set_tuning(exchange_grid=1)
            return small, full

        small, full = both(T.TERMS_ALL)
        assert _rel_err(small, S.apply(wl.X)).max() < TOL[prec]
        assert _rel_err(small, full).max() < tight
        small, full = both(T.TERM_K1D | T.TERM_D_EXX)
        assert _rel_err(small, S.apply(wl.X, T.TERM_K1D | T.TERM_D_EXX)).max() < TOL[prec]
        small, full = both(T.TERMS_ZVEC)
        assert _rel_err(small, S.apply(wl.X, T.TERMS_ZVEC)).max() < TOL[prec]
        assert _rel_err(small, full).max() < tight
        # stored tau live on the grid K1d runs on
        before = s.query()["device_bytes"]
        s.set_tuning(k1d_cache=1)
        assert s.query()["device_bytes"] - before == 36 * 64 ** 3 * (16 if prec == T.PREC_FP64 else 8)
        small, full = both(T.TERM_K1D)
        assert _rel_err(small, S.apply(wl.X, T.TERM_K1D)).max() < TOL[prec]
        assert _rel_err(small, full).max() < tight
        s.set_tuning(k1d_cache=0)
        assert s.query()["device_bytes"] == before
        s.close()


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_spin_flip(torch, prec):
    wl = _workload(24, 10.0, 10.0, 7, 3, seed=11, sf=True, nocc_tgt=5)
    want = O.system_from_workload(wl).apply(wl.X)
    got = _run(torch, wl, prec)
    assert _rel_err(got, want).max() < TOL[prec]


def test_ragged_tiles_give_the_same_result(torch):
    """Pair batches that do not divide the target and source counts."""
    wl = _workload(24, 10.0, 10.0, 11, 3, seed=12)
    want = O.system_from_workload(wl).apply(wl.X)
    for tiling in ((3, 5, 0, 0), (7, 2, 3, 1), (1, 1, 1, 0), (64, 16, 8, 1), (5, 3, 5, 1)):
        got = _run(torch, wl, T.PREC_FP64, tiling=tiling)
        assert _rel_err(got, want).max() < 1e-11, tiling
    got = _run(torch, wl, T.PREC_FP32, tiling=(4, 4, 4, 1))
    assert _rel_err(got, want).max() < 1e-5


@pytest.mark.parametrize("n,a,ecut", [(24, 10.0, 10.0), (72, 13.48, 25.0), (32, 9.0, 12.0), (64, 11.0, 25.0),
                                      (48, 10.0, 20.0)])
def test_kernel_variants_fp32(torch, n, a, ecut):
    """Every plane-pass variant (compact pair densities on / off, staged / register-resident /
    paired register z pass, loop / atomic accumulation, staged / register-line xy passes with one or
    two lanes per line) gives the
    oracle's L. The 24^3 grid aliases pair densities (pruning stays off there); 72^3, 64^3, 48^3 and
    32^3 do not (the register-line xy passes exist for 32, 48 and 64)."""
    wl = _workload(n, a, ecut, 6, 2, seed=15)
    want = O.system_from_workload(wl).apply(wl.X)
    for prune in (0, 1):
        for z in (0, 1, 2):
            for acc in (0, 1):
                for xy in (0, 1, 2, 3):
                    if xy != 0 and (prune == 0 or z == 0):
                        continue  # full planes: the xy passes are the staged ones whatever xy_kernel says
                    if xy in (2, 3) and acc == 0:
                        continue  # the loop accumulation runs the staged inverse pass
                    got = _run(torch, wl, T.PREC_FP32, tiling=dict(targets=3, sources=4, k1d_block=5,
                                                                  accumulate=acc, prune=prune, z_kernel=z,
                                                                  xy_kernel=xy))
                    assert _rel_err(got, want).max() < 1e-5, (prune, z, acc, xy)
    got = _run(torch, wl, T.PREC_FP64, tiling=(3, 4, 5, 1, -1, 1, 0))
    assert _rel_err(got, want).max() < 1e-11


@pytest.mark.parametrize("nocc", [20, 40, 100])
def test_k1d_all_pairs_and_blocks(torch, nocc):
    """K1d (Eq. 6) with the tau of every pair contracted in one pass (tuning.k1d_all = 1: FP32, compact
    intermediates on an alias-free grid, point-tiled tau; a ragged last orbital block, and odd block
    counts, where one block sits out each round of the pairing) and by 16 x 16 blocks of pairs
    (k1d_all = 0; also what k1d_all = 1 falls back to in FP64 and on the aliasing 24^3 grid), against
    the oracle."""
    for n, a, ecut in ((32, 9.0, 12.0), (24, 10.0, 10.0)):
        wl = _workload(n, a, ecut, nocc, 3, seed=40 + nocc)
        want = O.system_from_workload(wl).apply(wl.X, T.TERM_K1D)
        for prec in (T.PREC_FP32, T.PREC_FP64):
            for k1d_all in (1, 0):
                got = _run(torch, wl, prec, mask=T.TERM_K1D, tiling=dict(k1d_all=k1d_all))
                assert _rel_err(got, want).max() < TOL[prec], (n, prec, k1d_all)


def test_k1d_all_pairs_is_reproducible(torch):
    """The K1d term through the one-pass contraction sums in a fixed order (tau written once per
    point, one atomic add per output value and launch): two applications agree bit for bit, on a
    batch larger than one group of eight trial vectors."""
    wl = _workload(32, 9.0, 12.0, 40, 11, seed=44)
    s = T.system_from_workload(wl, precision=T.PREC_FP32, term_mask=T.TERM_K1D)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    first = s.apply(X).cpu().numpy()
    second = s.apply(X).cpu().numpy()
    s.close()
    assert np.array_equal(first, second)
    want = O.system_from_workload(wl).apply(wl.X, T.TERM_K1D)
    assert _rel_err(first.astype(np.complex128), want).max() < 1e-5


@pytest.mark.parametrize("sf", [False, True])
def test_init_from_device_inputs(torch, sf):
    """tddft_init_system with every input in device memory (CUDA tensors: orbitals of both spins,
    eigenvalues, V_loc, f_xc) builds the same operator as with host arrays, bit for bit (with the
    fixed-order accumulation: the atomic one sums in a different order from run to run)."""
    wl = _workload(24, 10.0, 10.0, 6, 2, seed=50, sf=sf, nocc_tgt=4 if sf else None)
    X = torch.from_numpy(wl.X).cuda()
    outs = []
    for dev in (False, True):
        put = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()) if dev else (lambda a: a)
        s = T.LiouvilleSystem(n=wl.n, a=wl.a, ecut=wl.ecut, phi_src=put(wl.phi_src), eps_src=put(wl.eps_src),
                              alpha=wl.alpha, kx_g0=wl.kx_g0, precision=T.PREC_FP64, nb_max=wl.nb,
                              spin_flip=wl.spin_flip, phi_tgt=put(wl.phi_tgt) if sf else None,
                              vloc=put(wl.vloc), fxc=put(wl.fxc))
        s.set_tuning(accumulate=0)
        outs.append(s.apply(X).cpu().numpy())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    want = O.system_from_workload(wl).apply(wl.X)
    assert _rel_err(outs[1], want).max() < TOL[T.PREC_FP64]


def test_projector_tensor_cores_match_simt(torch):
    """The tcgen05 projector (3xTF32 products, FP32 accumulation) against the SIMT
    FP32 projector and the oracle, on a batch whose rows exceed one 128-row tile."""
    wl = _workload(24, 10.0, 10.0, 40, 5, seed=16)
    want = O.system_from_workload(wl).apply(wl.X)
    tc = _run(torch, wl, T.PREC_FP32, tiling=(0, 0, 0, -1, -1, -1, -1, 1))
    staged = _run(torch, wl, T.PREC_FP32, tiling=(0, 0, 0, -1, -1, -1, -1, 2))
    simt = _run(torch, wl, T.PREC_FP32, tiling=(0, 0, 0, -1, -1, -1, -1, 0))
    assert _rel_err(tc, want).max() < 1e-5
    assert _rel_err(staged, want).max() < 1e-5
    assert _rel_err(tc, simt).max() < 2e-6
    assert _rel_err(tc, staged).max() < 1e-6  # the same products, packed or staged
    only_proj = _run(torch, wl, T.PREC_FP32, mask=T.TERM_D_KIN | T.TERM_PROJ, tiling=(0, 0, 0, -1, -1, -1, -1, 1))
    assert _rel_err(only_proj, O.system_from_workload(wl).apply(wl.X, T.TERM_D_KIN | T.TERM_PROJ)).max() < 1e-5


def test_tuning_fields_round_trip(torch):
    """Every writable field of tddft_tuning takes effect and reads back; -1 / 0 keep the value."""
    wl = _workload(24, 10.0, 10.0, 8, 2, seed=17)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    for kw in (dict(targets=4), dict(sources=2), dict(k1d_block=8), dict(accumulate=0), dict(accumulate=1),
               dict(graph=1), dict(graph=0), dict(prune=1), dict(prune=0), dict(z_kernel=0), dict(z_kernel=1),
               dict(z_kernel=2),
               dict(projector=0), dict(projector=2), dict(projector=1), dict(k1d_sparse=0), dict(k1d_sparse=1), dict(k1d_sparse=2),
               dict(k1d_cache=1), dict(k1d_cache=0), dict(exchange_grid=0), dict(exchange_grid=1),
               dict(xy_kernel=0), dict(xy_kernel=2), dict(xy_kernel=3), dict(xy_kernel=1),
               dict(k1d_all=0), dict(k1d_all=1)):
        before = s.get_tuning()
        s.set_tuning(**kw)
        after = s.get_tuning()
        (k, v), = kw.items()
        assert after[k] == v, (kw, after)
        assert {x: after[x] for x in after if x != k} == {x: before[x] for x in before if x != k}, (kw, before, after)
    with pytest.raises(T.TddftError):
        s.set_tuning(projector=3)
    with pytest.raises(T.TddftError):
        s.set_tuning(k1d_cache=2)
    with pytest.raises(T.TddftError):
        s.set_tuning(exchange_grid=2)
    with pytest.raises(T.TddftError):
        s.set_tuning(xy_kernel=4)
    s.close()


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
@pytest.mark.parametrize("n,a,ecut", [(24, 10.0, 10.0), (32, 9.0, 12.0)])
def test_stored_tau_give_the_recomputed_k1d(torch, prec, n, a, ecut):
    """K1d from the stored tau_vv' (tuning.k1d_cache) against the oracle and against the recomputing
    path, on 20 orbitals (a full 16-orbital block and a ragged 4-orbital one), with plain launches and
    under graph replay; the stored tau take the expected device memory and are released again. On
    24^3 (pair densities alias) they are stored block pair after block pair; on 32^3 in FP32 they are
    point-tiled and contracted in one pass."""
    wl = _workload(n, a, ecut, 20, 3, seed=18)
    want = O.system_from_workload(wl).apply(wl.X)
    want_k1d = O.system_from_workload(wl).apply(wl.X, T.TERM_K1D)
    s = T.system_from_workload(wl, precision=prec)
    Xd = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)
    plain = s.apply(Xd).cpu().numpy().astype(np.complex128)
    before = s.query()["device_bytes"]
    s.set_tuning(k1d_cache=1)
    fields = 16 * 16 + 16 * 4 + 4 * 4  # block pairs (0,0), (0,16), (16,16)
    assert s.query()["device_bytes"] - before == fields * n ** 3 * (16 if prec == T.PREC_FP64 else 8)
    got = s.apply(Xd).cpu().numpy().astype(np.complex128)
    assert _rel_err(got, want).max() < TOL[prec]
    assert _rel_err(got, plain).max() < (1e-13 if prec == T.PREC_FP64 else 1e-6)
    s.set_terms(T.TERM_K1D)
    assert _rel_err(s.apply(Xd).cpu().numpy().astype(np.complex128), want_k1d).max() < TOL[prec]
    s.set_terms(T.TERMS_ALL)
    s.set_tuning(graph=1)
    for _ in range(2):
        got_g = s.apply(Xd).cpu().numpy().astype(np.complex128)
        assert _rel_err(got_g, want).max() < TOL[prec]
    s.set_tuning(graph=0, k1d_cache=0)
    assert s.query()["device_bytes"] == before
    assert s.get_tuning()["k1d_cache"] == 0
    s.close()


def test_host_buffer_entry_point(torch):
    wl = _workload(24, 10.0, 10.0, 8, 4)
    want = O.system_from_workload(wl).apply(wl.X)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    got = s.apply_host(np.ascontiguousarray(wl.X.astype(np.complex64)))
    s.close()
    assert _rel_err(got.astype(np.complex128), want).max() < 1e-5


def test_hermiticity_fp32(torch):
    wl = _workload(24, 10.0, 10.0, 8, 2, seed=13)
    got = _run(torch, wl, T.PREC_FP32)
    lhs = np.vdot(wl.X[1], got[0])
    rhs = np.conj(np.vdot(wl.X[0], got[1]))
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_edge_cases(torch):
    wl = _workload(12, 7.0, 4.0, 3, 2)
    s = T.system_from_workload(wl, precision=T.PREC_FP64, nb_max=2)
    X = torch.from_numpy(wl.X).cuda()
    empty = torch.empty((0, 3, s.npw), dtype=torch.complex128, device="cuda")
    s.apply(empty)  # nb = 0 is a no-op
    with pytest.raises(T.TddftError) as e:
        s.apply(torch.cat([X, X]))  # nb > nb_max
    assert e.value.status == 1
    s.close()
    bad = wl.phi_src.copy()
    bad[0] *= 1.01
    with pytest.raises(T.TddftError) as e:
        T.LiouvilleSystem(n=12, a=7.0, ecut=4.0, phi_src=bad, eps_src=wl.eps_src, nb_max=1)
    assert e.value.status == 1
    with pytest.raises(T.TddftError):
        T.LiouvilleSystem(n=14, a=7.0, ecut=4.0, phi_src=wl.phi_src, eps_src=wl.eps_src, nb_max=1)


def test_alpha_zero_and_single_orbital(torch):
    wl = _workload(12, 7.0, 4.0, 1, 1, seed=14)
    wl.alpha = 0.0
    want = O.system_from_workload(wl).apply(wl.X)
    assert _rel_err(_run(torch, wl, T.PREC_FP64), want).max() < 1e-11


def test_diamond64_sampled_rows_fp32(torch):
    """64-atom diamond-like cell (72^3, 25 Ha, 128 orbitals, 8 trial vectors), the
    batch the benchmark times: every output checked on sampled rows (b, v)."""
    p = synth.WORKLOADS["diamond64"]
    wl = _workload(p["n"], 13.48, 25.0, 128, 8, seed=0)
    got = _run(torch, wl, T.PREC_FP32)
    rows = [(0, 0), (3, 77), (7, 127)]
    want = O.system_from_workload(wl).apply(wl.X, rows=rows)
    g = np.stack([got[b, v] for b, v in rows])
    assert _rel_err(g, want).max() < 1e-5
    # the same batch with K1d from the stored tau (27.5 GB)
    cached = _run(torch, wl, T.PREC_FP32, tiling=dict(k1d_cache=1))
    assert _rel_err(np.stack([cached[b, v] for b, v in rows]), want).max() < 1e-5
    assert _rel_err(cached, got).max() < 1e-6
    # every row lies in the unoccupied space
    ov = np.einsum("ug,bvg->buv", wl.phi_src.conj(), got)
    assert np.abs(ov).max() < 1e-5 * np.abs(got).max()
