"""The batched persistent form: many uneven FP32 cells in one launch.

Each cell of a batch is the same Hartree solve as a plan solve of that cell,
so the batched results are checked three ways:
  * against the FP64 oracle for the smaller cells (V_H rel L2 <= 2e-6, E_H rel <= 1e-7),
  * against plan solves of every cell of the 64-cell workload (same bars),
  * for determinism and CUDA-graph replay (bit-identical: every item does the
    same arithmetic whichever CTA takes it, and the E_H partials are summed in
    a fixed order).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1209_4506_gb300 import synth
from paper_1209_4506_gb300.hartree import HartreeBatch, HartreePlan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_V, TOL_E = 2e-6, 1e-7


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_batch(systems):
    B = HartreeBatch([(S.n, S.cell, S.sigma, S.pos.shape[0]) for S in systems])
    pos = torch.tensor(np.concatenate([S.pos for S in systems]).reshape(-1, 3), device="cuda")
    q = torch.tensor(np.concatenate([S.q for S in systems]), device="cuda")
    return B, pos, q


def test_offsets_concatenate_cells():
    systems = synth.config4()[:5]
    B, _, _ = make_batch(systems)
    sizes = [int(np.prod(S.n)) for S in systems]
    assert B.grid_off.tolist() == np.concatenate([[0], np.cumsum(sizes)]).tolist()
    assert B.atom_off.tolist() == np.concatenate([[0], np.cumsum([S.pos.shape[0] for S in systems])]).tolist()


def test_batched_matches_oracle_on_small_cells():
    O.set_threads(os.cpu_count() or 1)
    cells = sorted(synth.config4(), key=lambda S: np.prod(S.n))[:4]
    B, pos, q = make_batch(cells)
    vh, eh = B.solve(pos, q)
    B.device_status()
    for c, S in enumerate(cells):
        ref = O.solve_system(S, with_forces=False)
        v = B.cell_view(vh, c).cpu().numpy().astype(np.float64)
        assert rel_l2(v, ref["vh"]) <= TOL_V, S.name
        assert abs(eh[c].item() - ref["eh"]) <= TOL_E * abs(ref["eh"]), S.name


def test_batched_matches_plan_solves_on_64_uneven_cells():
    systems = synth.config4()
    B, pos, q = make_batch(systems)
    vh, eh = B.solve(pos, q)
    B.device_status()
    for c, S in enumerate(systems):
        plan = HartreePlan(S.n, S.cell, S.sigma, "fp32")
        v_ref, e_ref = plan.solve(torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda"))
        torch.cuda.synchronize()
        v = B.cell_view(vh, c)
        assert rel_l2(v.double().cpu().numpy(), v_ref.double().cpu().numpy()) <= TOL_V, S.name
        assert abs(eh[c].item() - e_ref.item()) <= TOL_E * abs(e_ref.item()), S.name
        plan.close()


def test_empty_and_single_atom_cells():
    cells = [
        synth.random_system((48, 48, 48), (8.0, 8.0, 8.0), 0, 0.6, seed=1, precision="fp32"),
        synth.random_system((64, 48, 40), (10.0, 8.0, 7.0), 1, 0.6, seed=2, precision="fp32", neutral=False),
        synth.random_system((96, 80, 72), (16.0, 13.6, 12.0), 200, 0.6, seed=3, precision="fp32"),
    ]
    B, pos, q = make_batch(cells)
    vh, eh = B.solve(pos, q)
    B.device_status()
    assert eh[0].item() == 0.0 and torch.count_nonzero(B.cell_view(vh, 0)).item() == 0
    O.set_threads(os.cpu_count() or 1)
    for c in (1, 2):
        ref = O.solve_system(cells[c], with_forces=False)
        assert rel_l2(B.cell_view(vh, c).double().cpu().numpy(), ref["vh"]) <= TOL_V
        assert abs(eh[c].item() - ref["eh"]) <= TOL_E * abs(ref["eh"])


def test_repeat_is_bit_identical():
    systems = synth.config4()[:16]
    B, pos, q = make_batch(systems)
    v1, e1 = B.solve(pos, q)
    v1, e1 = v1.clone(), e1.clone()
    v2, e2 = B.solve(pos, q)
    B.device_status()
    assert torch.equal(v1, v2) and torch.equal(e1, e2)


def test_cuda_graph_capture_and_replay():
    systems = synth.config4()[:16]
    B, pos, q = make_batch(systems)
    vh = torch.empty(int(B.grid_off[-1]), dtype=torch.float32, device="cuda")
    eh = torch.empty(len(systems), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.solve(pos, q, vh, eh)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.solve(pos, q, vh, eh)
    # new positions written into the captured input buffer, then replay
    rng = np.random.default_rng(5)
    cells = [np.asarray(S.cell) for S in systems]
    new = np.concatenate([S.pos + rng.normal(0.0, 0.05, S.pos.shape) for S in systems])
    new = np.concatenate([synth.wrap(new[B.atom_off[c]:B.atom_off[c + 1]], tuple(cells[c]))
                          for c in range(len(systems))])
    pos.copy_(torch.tensor(new, device="cuda"))
    g.replay()
    torch.cuda.synchronize()
    B.device_status()
    v_ref, e_ref = B.solve(pos, q)
    torch.cuda.synchronize()
    assert torch.equal(vh, v_ref) and torch.equal(eh, e_ref)


def test_injected_lost_producer_times_out_and_the_next_solve_is_correct():
    """Failure detection without a GPU fault: one producer item (stage 4, the c pass, of cell 1)
    is told never to report itself done, and the dependency waits get a short limit.  The
    items of the next stage of that cell wait, give up and set the batch's error word; the
    host reads HARTREE_ERR_TIMEOUT.  The context stays usable: with the injection switched
    off, the next solve on the same batch matches the oracle."""
    from paper_1209_4506_gb300 import capi

    O.set_threads(os.cpu_count() or 1)
    cells = sorted(synth.config4(), key=lambda S: np.prod(S.n))[:3]
    B, pos, q = make_batch(cells)
    with pytest.raises(capi.HartreeError):
        B.fault_inject(skip_stage=9, skip_cell=0)  # the E_H sum has no successor: refused
    with pytest.raises(capi.HartreeError):
        B.fault_inject(skip_stage=4, skip_cell=len(cells))
    B.fault_inject(skip_stage=4, skip_cell=1, spin_limit=2000)  # about 0.1 ms per wait
    vh, eh = B.solve(pos, q)
    with pytest.raises(capi.HartreeError) as ei:
        B.device_status()
    assert ei.value.status == capi.HARTREE_ERR_TIMEOUT
    B.device_status()  # the error word was cleared by the check
    B.fault_inject(-1)
    vh, eh = B.solve(pos, q)
    B.device_status()
    for c, S in enumerate(cells):
        ref = O.solve_system(S, with_forces=False)
        v = B.cell_view(vh, c).cpu().numpy().astype(np.float64)
        assert rel_l2(v, ref["vh"]) <= TOL_V, S.name
        assert abs(eh[c].item() - ref["eh"]) <= TOL_E * abs(ref["eh"]), S.name
