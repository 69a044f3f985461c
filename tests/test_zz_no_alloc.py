"""hedl_eval_concept_noalloc: the evaluation entry point for callers that may
not allocate device memory when they evaluate (so cannot hand over the
workspace hedl_eval_concept wants).  It uses the library's built-in scratch
array; its results must equal hedl_eval_concept's, call after call.

Kept in a file of its own, collected last, so that a run stopping at the
first failure has run every other test before it."""
import numpy as np
import pytest

import paper_2412_00802_gb300 as H
from synth import hyps, kb as K, programs as P
from synth.rng import Rng
from tests import oracle_pins as pins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dkb():
    import torch
    from paper_2412_00802_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    kb = K.generate(K.CONFIGS["small"])
    return kb, H.DeviceKB.from_synth(kb)


def test_no_alloc_matches_eval_concept_on_two_calls(dkb):
    import torch
    kb, d = dkb
    r = Rng(12, 12)
    progs = [np.array(pins.random_program(r, kb, r.randint(1, 6)).postfix(), np.uint64) for _ in range(24)]
    progs += hyps.batch_hyps(kb, 13, 0, 8)
    import oracle
    okb = oracle.from_synth(kb)
    for prog in progs:
        want = d.eval(prog)                                  # the existing entry point, caller workspace
        # and the instance set itself, from the independent CPU evaluator
        assert np.array_equal(K.unpack_bits(want, kb.n), oracle.eval_program(okb, prog))
        for call in range(2):                                # two calls in a row on the shared scratch
            out = torch.full((d.wp,), -1, dtype=torch.int32, device="cuda")
            H.hedl_eval_concept_noalloc(d.handle, prog, out)
            H.hedl_sync_status(d.handle)
            got = out.cpu().numpy().view(np.uint32)
            assert np.array_equal(got, want), (call, P.to_text(P.from_postfix(prog)))


def test_no_alloc_rejects_programs_beyond_the_scratch(dkb):
    import torch
    kb, d = dkb
    # a chain of nested EXISTS: every filler is a materialized row, about
    # 16,000 rows of 1,264 bytes > 16 MiB
    chain = [P.insn(P.ATOM, 0, 1)] + [P.insn(P.EXISTS, 0, 0)] * 16_000
    out = torch.zeros(d.wp, dtype=torch.int32, device="cuda")
    with pytest.raises(H.HedlError) as e:
        H.hedl_eval_concept_noalloc(d.handle, np.array(chain, np.uint64), out)
    assert e.value.code == -3 and "built-in scratch" in e.value.msg
