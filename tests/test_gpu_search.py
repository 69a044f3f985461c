"""The refinement beam search on the GPU against the oracle's exhaustive
search, and the surrogate-ordered search without pruning against the
exhaustive one (identical final beams)."""
import numpy as np
import pytest

import oracle
from oracle import search as OS
from synth import kb as K, programs as P
from synth.refine import Refiner

pytestmark = pytest.mark.gpu


def _refine_fn(refiner):
    def f(beam_progs, step, count):
        nodes = [P.from_postfix(p) for p in beam_progs]
        return [np.array(n.postfix(), np.uint64) for n in refiner.refine(nodes, step, count)]
    return f


@pytest.fixture(scope="module")
def env():
    from paper_2412_00802_gb300 import build
    build.build()
    import paper_2412_00802_gb300 as H
    kb = K.generate(K.CONFIGS["search"].scaled(20000, n_concepts=40, n_roles=8, n_props=6))
    return H, kb, H.DeviceKB.from_synth(kb)


def test_exhaustive_search_matches_oracle(env):
    H, kb, dkb = env
    from paper_2412_00802_gb300.search import BeamSearch
    ref = Refiner(kb, 77)
    start = [np.array(n.postfix(), np.uint64) for n in ref.start()]
    beam, logs = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512, batch=200).run(start, 4)
    want = OS.exhaustive(oracle.from_synth(kb), _refine_fn(ref), start, 4, 16, 512)
    got = [(e.prog.tobytes(), e.counts) for e in beam]
    assert got == want
    assert logs[-1].best_acc >= logs[0].best_acc


def test_surrogate_order_without_pruning_keeps_the_beam(env):
    H, kb, dkb = env
    from paper_2412_00802_gb300.search import BeamSearch
    from paper_2412_00802_gb300.surrogate import Surrogate
    ref = Refiner(kb, 78)
    start = [np.array(n.postfix(), np.uint64) for n in ref.start()]
    plain, _ = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512).run(start, 3)
    ordered, logs = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512, surrogate=Surrogate(seed=3)).run(start, 3)
    assert [(e.prog.tobytes(), e.counts) for e in plain] == [(e.prog.tobytes(), e.counts) for e in ordered]
    # trained online on its own exact scores, still without pruning: the same beam
    online, _ = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512, surrogate=Surrogate(seed=3),
                           online_epochs=2).run(start, 3)
    assert [(e.prog.tobytes(), e.counts) for e in plain] == [(e.prog.tobytes(), e.counts) for e in online]
    pruned, plog = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512, surrogate=Surrogate(seed=3),
                              keep_fraction=0.25, online_epochs=2, warmup_steps=1).run(start, 3)
    assert plog[0].evaluated == plog[0].candidates          # the warm-up step scores everything
    assert all(l.evaluated <= 0.26 * l.candidates + 1 for l in plog[1:])
    adaptive, alog = BeamSearch(dkb, _refine_fn(ref), width=16, per_step=512, batch=64, surrogate=Surrogate(seed=3),
                                adaptive=True, online_epochs=2, warmup_steps=1).run(start, 3)
    assert alog[0].evaluated == alog[0].candidates
    assert all(1 <= l.evaluated <= l.candidates for l in alog)
    # every reported score is exact
    okb = oracle.from_synth(kb)
    for e in pruned + adaptive:
        c, _, _ = oracle.eval_batch(okb, e.prog, np.array([0, len(e.prog)]))
        assert tuple(int(x) for x in c[0]) == e.counts
