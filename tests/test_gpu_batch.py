"""Batches and the autotuner on the GPU, through the C ABI.

A batch advances many independent simulations with one launch per stage; each
member must compute exactly what it computes alone:
* strict build: after one batched step every member's cells, offsets, momenta
  and tile_offset equal the FP32 oracle bit for bit (members of different
  grid sizes, tile sizes, species counts and CTA splits in one batch);
* multi-step: the energies of each member follow its own single-simulation
  run within FP32 round-off (the J flush adds in a different order);
* a member stepped, reloaded or re-tiled on its own, or destroyed, is picked
  up by the next batched step;
* the autotuner leaves the simulation's state where it found it and its
  choice steps like any other tiling.
"""
import numpy as np
import pytest

import oracle
from paper_2501_14795_gb300 import pic
from paper_2501_14795_gb300 import workloads as wl
from test_gpu_parity import (F_RTOL, J_RTOL, _by_id, _gpu, _oracle, _oracle_by_id,
                             _random_case, _tile_ids)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_14795_gb300 import build
    build.build_library()
    oracle.build_oracle()


def _members():
    """(workload, E, B, tile, chunk, threads) of a mixed batch."""
    out = []
    for (nx, ny, T, n, chunk, threads) in [(48, 32, 16, 5003, 0, 256), (64, 64, 8, 20011, 0, 128),
                                            (32, 64, 32, 7001, 0, 256), (64, 32, 16, 9000, 64, 64),
                                            (16, 16, 8, 0, 0, 256)]:
        w, E, B = _random_case(nx, ny, T, n, seed=nx * 7 + ny + T + n)
        out.append((w, E, B, T, chunk, threads))
    # two species on one grid
    w2 = wl.two_stream(nx=64, ny=32, k=2, u_th=0.1, drift=0.3, tile=16, seed=5)
    sp_b = wl.random_particles(64, 32, 3000, u_max=0.5, seed=77, q_over_m=1.0, qtilde=1.0 / 8)
    w2.species.append(sp_b)
    E2, B2 = wl.random_fields(64, 32, amp=0.1, seed=6)
    out.append((w2, E2, B2, 16, 0, 256))
    return out


def _build(members, flags):
    sims = []
    for (w, E, B, T, chunk, threads) in members:
        sims.append(_gpu(w, flags, tile=T, threads=threads, E=E, B=B, chunk=chunk))
    return sims


def test_one_batched_step_is_bit_exact_with_fp32_oracle():
    members = _members()
    sims = _build(members, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS)
    try:
        with pic.Batch(sims) as b:
            b.step(1)
            b.sync()
            tot, per = b.kernel_launches()
            assert tot == per and per >= 6
        for (w, E, B, T, chunk, threads), sim in zip(members, sims):
            o32 = _oracle(w, np.float32, E, B, T)
            o32.step(1)
            o64 = _oracle(w, np.float64, E, B, T)
            o64.step(1)
            for k, sp in enumerate(o32.species):
                got = sim.particles(k, ids=True)
                g = _by_id(got)
                ref = _oracle_by_id(sp)
                for key in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
                    np.testing.assert_array_equal(g[key], ref[key], err_msg=f"{w.name} s{k} {key}")
                np.testing.assert_array_equal(got["tile_offset"], o32.tile_offsets(k))
                tid = _tile_ids(got["ix"], got["iy"], w.nx, T)
                off = got["tile_offset"]
                assert all(np.all(tid[off[t]:off[t + 1]] == t) for t in range(len(off) - 1))
            Jg = sim.fields(pic.FIELD_J)
            J64 = o64.J
            scale = max(np.abs(J64).max(), 1e-30)
            assert np.abs(Jg - J64).max() <= J_RTOL * scale + 1e-30, w.name
            for which, ref in ((pic.FIELD_E, o64.E), (pic.FIELD_B, o64.B)):
                got = sim.fields(which)
                assert np.abs(got - ref).max() <= F_RTOL * max(np.abs(ref).max(), 1e-3), w.name
            d = sim.diagnostics()
            assert d["status_bits"] == 0 and d["step"] == 1
    finally:
        for s in sims:
            s.close()


def _energies(sim, steps):
    we, wb, wk = sim.history(0, steps + 1)
    return np.asarray(we), np.asarray(wb), np.asarray(wk[:steps])


def test_batched_steps_follow_single_runs():
    members = _members()
    steps = 40
    alone = _build(members, pic.PIC_TRACK_IDS)
    batched = _build(members, pic.PIC_TRACK_IDS)
    try:
        for s in alone:
            s.step(steps)
        with pic.Batch(batched) as b:
            b.step(steps)
            b.sync()
            tot, per = b.kernel_launches()
            assert tot == steps * per
        for (w, *_), a, s in zip(members, alone, batched):
            da, ds = a.diagnostics(), s.diagnostics()
            assert ds["status_bits"] == 0 and ds["step"] == steps
            assert da["n_particles"] == ds["n_particles"]
            ea, eb = _energies(a, steps), _energies(s, steps)
            for x, y in zip(ea, eb):
                np.testing.assert_allclose(y, x, rtol=2e-3, atol=1e-7, err_msg=w.name)
            # the random initial fields break Gauss's law; the residual is carried along
            np.testing.assert_allclose(ds["gauss_max"], da["gauss_max"], rtol=1e-3, err_msg=w.name)
    finally:
        for s in alone + batched:
            s.close()


def test_batch_picks_up_member_changes():
    """Stepping one member alone, re-tiling another and destroying a third
    between batched steps: the batch rebuilds and keeps every member right."""
    members = _members()[:4]
    ref = _build(members, pic.PIC_TRACK_IDS)
    sims = _build(members, pic.PIC_TRACK_IDS)
    try:
        b = pic.Batch(sims)
        b.step(3)
        sims[1].step(2)           # member 1 alone
        sims[2].set_tiling(16)    # member 2: T 32 -> 16
        b.step(3)
        gone = sims.pop(3)
        gone.close()              # leaves the batch
        b.step(2)
        b.sync()
        b.close()
        for s in ref[:3]:
            s.step(8)
        ref[1].step(2)
        for (w, *_), r, s in zip(members, ref, sims):
            dr, ds = r.diagnostics(), s.diagnostics()
            assert ds["step"] == dr["step"] and ds["status_bits"] == 0
            np.testing.assert_allclose(ds["w_e"], dr["w_e"], rtol=2e-3, atol=1e-8, err_msg=w.name)
            np.testing.assert_allclose(ds["w_k"], dr["w_k"], rtol=1e-5, err_msg=w.name)
        assert sims[2].num_tiles() == (32 // 16) * (64 // 16)
    finally:
        for s in ref + sims:
            s.close()


def test_batch_rejects_bad_members():
    members = _members()[:2]
    a, b_ = _build(members, pic.PIC_TRACK_IDS)
    strict = _build(members[:1], pic.PIC_STRICT_FP)[0]
    try:
        with pytest.raises(pic.PicError):
            pic.Batch([a, a])
        with pytest.raises(pic.PicError):
            pic.Batch([a, strict])
        with pic.Batch([a, b_]):
            with pytest.raises(pic.PicError):
                pic.Batch([b_])   # already in a batch
        pic.Batch([b_]).close()   # free again once the first batch is gone
    finally:
        for s in (a, b_, strict):
            s.close()


def test_autotune_restores_state_and_steps_like_any_tiling():
    w = wl.two_stream(nx=64, ny=64, k=4, u_th=0.1, drift=0.2, tile=16, seed=3)
    with _gpu(w, pic.PIC_TRACK_IDS) as sim, _gpu(w, pic.PIC_TRACK_IDS) as ref:
        sim.step(5)
        ref.step(5)
        before = _by_id(sim.particles(0, ids=True))
        E0 = sim.fields(pic.FIELD_E)
        d0 = sim.diagnostics()
        T, n, ms = sim.autotune(steps=3, force=True)
        assert T in (8, 16, 32) and n in (64, 128, 256, 512) and ms > 0
        after = _by_id(sim.particles(0, ids=True))
        for k in ("id", "ix", "iy", "x", "y", "ux", "uy", "uz"):
            np.testing.assert_array_equal(after[k], before[k], err_msg=k)
        np.testing.assert_array_equal(sim.fields(pic.FIELD_E), E0)
        d1 = sim.diagnostics()
        assert d1["step"] == d0["step"] and d1["w_e"] == d0["w_e"] and d1["w_k"] == d0["w_k"]
        assert sim.num_tiles() == (64 // T) ** 2
        sim.step(10)
        ref.step(10)
        ds, dr = sim.diagnostics(), ref.diagnostics()
        assert ds["status_bits"] == 0
        np.testing.assert_allclose(ds["w_k"], dr["w_k"], rtol=1e-5)
        np.testing.assert_allclose(ds["w_e"], dr["w_e"], rtol=1e-3, atol=1e-9)
        # a second call with the same key takes the cached choice without timing
        T2, n2, ms2 = sim.autotune(steps=3)
        assert (T2, n2, ms2) == (T, n, 0.0)


def test_set_tiling_resorts_particles():
    w, E, B = _random_case(64, 64, 16, 12000, seed=4242)
    with _gpu(w, pic.PIC_STRICT_FP | pic.PIC_TRACK_IDS, tile=16, E=E, B=B) as sim:
        sim.set_tiling(8, 128)
        assert sim.num_tiles() == 64
        sim.step(1)
        got = sim.particles(0, ids=True)
    o32 = _oracle(w, np.float32, E, B, 8)
    o32.step(1)
    g, ref = _by_id(got), _oracle_by_id(o32.species[0])
    for k in ("ix", "iy", "x", "y", "ux", "uy", "uz"):
        np.testing.assert_array_equal(g[k], ref[k], err_msg=k)
    np.testing.assert_array_equal(got["tile_offset"], o32.tile_offsets())
    with _gpu(w, 0, tile=16) as sim:
        with pytest.raises(pic.PicError):
            sim.set_tiling(12)
