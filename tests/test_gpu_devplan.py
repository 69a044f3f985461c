"""Plans built on the device (hedl_plan_batch_device; the paper's future work, Section VII):
the image equals the host planner's without sharing or slicing, byte for byte, and the plan
runs bit-exact against the oracle."""
import numpy as np
import pytest

import oracle
import paper_2412_00802_gb300 as H
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import oracle_pins as pins
from tests.gpu_util import THREADS, device_kb

pytestmark = pytest.mark.gpu

F = H.HEDL_NO_CSE | H.HEDL_NO_SLICE


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_00802_gb300 import build
    build.build()
    oracle.build()


def _device_plan(dkb, flat, offs, flags=0):
    import torch
    pd = torch.from_numpy(np.ascontiguousarray(flat).view(np.int64)).to(dkb.device)
    od = torch.from_numpy(np.ascontiguousarray(offs, np.uint32).view(np.int32)).to(dkb.device)
    return H.hedl_plan_batch_device(dkb.handle, pd, od, int(offs[-1]), flags)


@pytest.fixture(scope="module")
def mixed():
    kb = K.generate(K.CONFIGS["small"].scaled(3000, seed=5, n_num_roles=2, n_str_roles=2, n_strings=50,
                                              n_patterns=6))
    return kb, device_kb(kb)


@pytest.mark.parametrize("stage", [0, 1])
def test_device_plan_image_equals_the_host_planners(mixed, stage):
    """Random batches over every construct (numeric and string roles included), deep chains that
    force materialisation, per-level launches: the device-built image is the host planner's
    (HEDL_NO_CSE | HEDL_NO_SLICE) byte for byte, and the plan info agrees field by field."""
    kb, dkb = mixed
    H.hedl_tuning_set(dkb.handle, stage_fillers=stage)
    r = Rng(5, 17)
    try:
        for it in range(16):
            progs = [np.array(pins.random_program(r, kb, r.randint(1, 9)).postfix(), np.uint64)
                     for _ in range(r.randint(1, 300))]
            if it % 5 == 0:
                progs.append(np.array([P.insn(P.ATOM, 0, 0)] + [x for i in range(200) for x in (
                    P.insn(P.ATOM, 0, i % kb.n_concepts), P.insn(P.AND if i % 2 else P.OR))], np.uint64))
                progs.append(np.array([P.insn(P.ATOM, 0, 2)] + [P.insn(P.EXISTS, 0, it % kb.n_roles)] * 300,
                                      np.uint64))
            if it % 3 == 0:
                progs += hyps.small_hyps(kb, it, 400)
            flat, offs = P.pack_batch(progs)
            for extra in (0, H.HEDL_LEVELS):
                a = H.hedl_plan_batch(dkb.handle, flat, offs, F | extra)
                b = _device_plan(dkb, flat, offs, extra)
                assert np.array_equal(H.hedl_plan_image(a), H.hedl_plan_image(b)), (it, extra)
                assert H.hedl_plan_info_get(a) == H.hedl_plan_info_get(b), (it, extra)
    finally:
        H.hedl_tuning_set(dkb.handle, stage_fillers=0)


def test_device_plan_runs_bit_exact(mixed):
    """A device-built plan, executed (its image copied within the device) and replayed, gives the
    oracle's instance sets and counts."""
    import torch
    kb, dkb = mixed
    progs = hyps.small_hyps(kb, 3, 700)
    r = Rng(8, 2)
    progs += [np.array(pins.random_program(r, kb, r.randint(1, 8)).postfix(), np.uint64) for _ in range(300)]
    flat, offs = P.pack_batch(progs)
    okb = oracle.from_synth(kb)
    oc, osets, errs = oracle.eval_batch(okb, flat, offs, threads=THREADS, keep_sets=True)
    assert not errs.any()
    for extra in (0, H.HEDL_LEVELS):
        plan = _device_plan(dkb, flat, offs, extra)
        ws = dkb.workspace(H.hedl_plan_info_get(plan)["workspace_bytes"])
        for call in (H.hedl_plan_execute, H.hedl_plan_replay, H.hedl_plan_execute):
            counts = torch.zeros((len(progs), 4), dtype=torch.int32, device=dkb.device)
            bits = torch.zeros((len(progs), dkb.wp), dtype=torch.int32, device=dkb.device)
            call(dkb.handle, plan, counts, bits, ws)
            H.hedl_sync_status(dkb.handle)
            assert np.array_equal(counts.cpu().numpy().astype(np.int64), oc), (extra, call.__name__)
            bb = bits.cpu().numpy().view(np.uint32)
            for h in range(len(progs)):
                assert np.array_equal(K.unpack_bits(bb[h], kb.n), osets[h].astype(bool)), (extra, h)


def test_device_planner_rejects_bad_input(mixed):
    """Validation on the device names the first bad program (as hedl_plan_batch does); offsets
    outside the instruction array are refused before any scratch is indexed; a chain deeper than
    the sort key's 2^14 levels is refused."""
    import torch
    kb, dkb = mixed
    progs = hyps.small_hyps(kb, 1, 10)
    progs[6] = np.array([P.insn(P.OR)], np.uint64)
    flat, offs = P.pack_batch(progs)
    with pytest.raises(H.HedlError) as e:
        _device_plan(dkb, flat, offs)
    assert e.value.code == -2 and "program 6" in str(e.value)
    progs[6] = np.array([P.insn(P.ATOM, 0, kb.n_concepts)], np.uint64)   # concept id out of range
    with pytest.raises(H.HedlError) as e:
        _device_plan(dkb, *P.pack_batch(progs))
    assert e.value.code == -2 and "program 6" in str(e.value)
    good = hyps.small_hyps(kb, 1, 10)
    flat, offs = P.pack_batch(good)
    bad_offs = offs.copy()
    bad_offs[4] = bad_offs[-1] + 50                                       # past the instructions
    pd = torch.from_numpy(flat.view(np.int64)).to(dkb.device)
    od = torch.from_numpy(bad_offs.astype(np.uint32).view(np.int32)).to(dkb.device)
    with pytest.raises(H.HedlError) as e:
        H.hedl_plan_batch_device(dkb.handle, pd, od, int(offs[-1]))
    assert e.value.code == -1
    with pytest.raises(H.HedlError) as e:                                  # n_insns disagrees with offs
        H.hedl_plan_batch_device(dkb.handle, pd, torch.from_numpy(offs.astype(np.uint32).view(np.int32)).to(dkb.device),
                                 int(offs[-1]) - 1)
    assert e.value.code == -1
    chain = [P.insn(P.ATOM, 0, 1)] + [P.insn(P.EXISTS, 0, 0)] * 17_000
    with pytest.raises(H.HedlError) as e:
        _device_plan(dkb, *P.pack_batch([np.array(chain, np.uint64)]))
    assert e.value.code == -1 and "16,384 dependency levels" in str(e.value)
    for bad_flags in (H.HEDL_PLAIN, H.HEDL_SLICE_ALL):
        with pytest.raises(H.HedlError) as e:
            _device_plan(dkb, flat, offs, bad_flags)
        assert e.value.code == -1


def test_device_plan_on_the_bench_batch():
    """The 4,096-hypothesis batch of the batched workload's shape (on a 200,000-individual KB of
    its distributions): same image as the host planner, counts equal the host plan's."""
    import torch
    kb = K.generate(K.CONFIGS["batch"].scaled(200_000))
    dkb = device_kb(kb)
    gen = hyps.TreeGen(kb, 1003, share=0.3)
    flat, offs = P.pack_batch(hyps.batch_hyps(kb, 1003, 3, 4096, gen=gen))
    a = H.hedl_plan_batch(dkb.handle, flat, offs, F)
    b = _device_plan(dkb, flat, offs)
    assert np.array_equal(H.hedl_plan_image(a), H.hedl_plan_image(b))
    ws = dkb.workspace(H.hedl_plan_info_get(a)["workspace_bytes"])
    got = []
    for plan in (a, b):
        counts = torch.zeros((4096, 4), dtype=torch.int32, device=dkb.device)
        H.hedl_plan_execute(dkb.handle, plan, counts, None, ws)
        H.hedl_sync_status(dkb.handle)
        got.append(counts.cpu().numpy())
    assert np.array_equal(got[0], got[1])
