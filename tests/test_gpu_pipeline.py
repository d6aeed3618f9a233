"""Host-buffer stepping with two contexts in turn (the end-to-end pattern):
state set from pinned host memory without waiting, a CFL step, the result
read back; each context's step ordered after the other's by an event.  Every
result must equal, to the bit, that of one context stepping the same inputs
one after the other."""
import numpy as np
import pytest

from paper_2511_20337_b300 import mhd
from paper_2511_20337_b300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def inputs(cfg, st, count):
    """count different pinned host states: the base state with a seeded
    density perturbation (energy adjusted to keep the pressure positive)."""
    rng = np.random.default_rng(3)
    out = []
    for _ in range(count):
        s = {k: np.array(v) for k, v in st.items()}
        f = 1.0 + 0.01 * rng.standard_normal(s["rho"].shape)
        s["rho"] = s["rho"] * f
        s["E"] = s["E"] * f
        out.append({k: torch.from_numpy(v).pin_memory() for k, v in s.items()})
    return out


@pytest.mark.parametrize("case", ["turbulent3d-48", "ensemble-batch"])
def test_two_contexts_in_turn_equal_one_context(case):
    dev = torch.device("cuda", 0)
    nsteps = 6
    if case == "turbulent3d-48":
        cfg, st = W.turbulent_3d(48)
        ins = inputs(cfg, st, nsteps)
        ref = mhd.Sim(cfg)
        want = []
        for h in ins:
            ref.set_conserved(h)
            ref.advance(1)
            want.append(ref.get_conserved())
        streams = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))
        ctxs = [mhd.Sim(cfg, stream=s.cuda_stream) for s in streams]
        outs = [{k: torch.empty_like(v).pin_memory() for k, v in ins[0].items()} for _ in range(nsteps)]
        prev, done = None, None
        for s in range(nsteps):
            c, cs = ctxs[s % 2], streams[s % 2]
            c.set_conserved(ins[s])
            if done is not None:
                cs.wait_event(done)
            c.advance(1)
            done = torch.cuda.Event()
            done.record(cs)
            if prev is not None:
                prev[0].get_conserved(outs[prev[1]])
            prev = (c, s)
        prev[0].get_conserved(outs[prev[1]])
        for s in range(nsteps):
            for k in want[s]:
                assert np.array_equal(outs[s][k].numpy(), want[s][k]), (s, k)
    else:
        members = W.ensemble_members(6, seed=9, sizes=(32, 48, 64))
        cases = [W.ensemble_member_state(m) for m in members]
        cfgs = [c for c, _ in cases]
        runs = [inputs(c, s, 3) for c, s in cases]
        ref = mhd.Batch(cfgs)
        want = []
        for t in range(3):
            for r in range(len(cases)):
                ref.set_conserved(r, runs[r][t])
            ref.step(1)
            want.append([ref.get_conserved(r) for r in range(len(cases))])
        streams = (torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev))
        bts = [mhd.Batch(cfgs, stream=s.cuda_stream) for s in streams]
        got = [[None] * len(cases) for _ in range(3)]
        prev, done = None, None
        for t in range(3):
            b, bs = bts[t % 2], streams[t % 2]
            for r in range(len(cases)):
                b.set_conserved(r, runs[r][t])
            if done is not None:
                bs.wait_event(done)
            b.step(1)
            done = torch.cuda.Event()
            done.record(bs)
            if prev is not None:  # queued read-outs into pinned buffers, one wait
                pb, pt = prev
                got[pt] = [{k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in want[pt][r].items()}
                           for r in range(len(cases))]
                for r in range(len(cases)):
                    pb.get_conserved(r, got[pt][r], wait=False)
                pb.synchronize()
                got[pt] = [{k: v.numpy() for k, v in d.items()} for d in got[pt]]
            prev = (b, t)
        got[prev[1]] = [prev[0].get_conserved(r) for r in range(len(cases))]
        for t in range(3):
            for r in range(len(cases)):
                for k in want[t][r]:
                    assert np.array_equal(got[t][r][k], want[t][r][k]), (t, r, k)
