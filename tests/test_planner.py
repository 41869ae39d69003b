"""CPU tests of the optimizer (no GPU): the plan, run by the numpy plan
interpreter, must equal the oracle's unoptimised gate-by-gate result; plus
structural properties of the diagonal detector (Algorithm 8), the gate-block
search and the fusion."""
import numpy as np
import pytest

import oracle
from paper_2604_12256_gb300 import circuits as C
from paper_2604_12256_gb300 import svsim as S
from plan_interp import interpret

pytestmark = pytest.mark.usefixtures("built_lib")

FLAG_SETS = {
    "unfused": 0,
    "diag": S.SIM_F_DIAG,
    "block": S.SIM_F_BLOCK,
    "block_fuse": S.SIM_F_BLOCK | S.SIM_F_FUSE,
    "all": S.SIM_F_DIAG | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_BOOST,
}

CIRCUITS = {
    "mixed": lambda n: C.random_mixed(n, 120, 100 + n, max_k=3),
    "layered": lambda n: C.layered(n, 6, n),
    "diagheavy": lambda n: C.diag_heavy(n, 150, n),
    "qft": lambda n: C.qft(n, n),
    "qaoa": lambda n: C.qaoa(n if n % 2 == 0 else n - 1, 2, n),
    "rzzfull": lambda n: C.rzz_full(n, n),
}


@pytest.mark.parametrize("flags", list(FLAG_SETS))
@pytest.mark.parametrize("name", list(CIRCUITS))
@pytest.mark.parametrize("n", [10, 13])
def test_plan_is_exact_c128(name, flags, n):
    c = CIRCUITS[name](n)
    opt = S.default_options(flags=FLAG_SETS[flags])
    plan = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, opt)
    got = interpret(plan, basis=c.basis)
    exp = oracle.run(c)
    np.testing.assert_allclose(got, exp, atol=1e-12, rtol=0)


@pytest.mark.parametrize("name", ["mixed", "diagheavy", "qft", "qaoa"])
def test_plan_is_exact_c64_weights(name):
    c = CIRCUITS[name](12)
    plan = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis)
    got = interpret(plan, basis=c.basis)
    exp = oracle.run(c)
    # 32-bit phase weights: <= 2^-33 turn per term
    np.testing.assert_allclose(got, exp, atol=2e-7, rtol=0)


def test_small_registers_fall_back_to_gate_by_gate():
    for n in (1, 3, 8):
        c = C.random_mixed(n, 40, n, max_k=min(3, n))
        plan = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis)
        assert all(op["op"] in ("gate", "phase") for op in plan["ops"])
        np.testing.assert_allclose(interpret(plan, basis=c.basis), oracle.run(c), atol=2e-7)


def test_blocking_cuts_sweeps():
    c = C.diag_heavy(20, 500, 1)
    unf = S.plan_json(c.n, c.gates, S.SIM_C64, 0, S.default_options(flags=0))
    blk = S.plan_json(c.n, c.gates, S.SIM_C64, 0)
    assert unf["stats"]["gates_in"] == 520
    assert blk["stats"]["sweeps"] * 10 < unf["stats"]["ops"]


def test_qft_needs_few_sweeps():
    c = C.qft(30, 2)
    p = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis)
    assert p["stats"]["sweeps"] <= 8, p["stats"]


def test_diagonal_detector_fuses_across_barriers():
    # diagonals separated by non-diagonal gates on other qubits (barriers that
    # do not touch the fused set) fuse into ONE diagonal; a naive scan that
    # stops at every non-diagonal gate would produce three.
    g = [C.Gate("rzz", (0, 1), (0.3,)), C.Gate("h", (2,)), C.Gate("ry", (3,), (0.2,)),
         C.Gate("rzz", (1, 4), (0.5,)), C.Gate("cp", (0, 4), (0.7,)), C.Gate("rx", (2,), (0.4,)),
         C.Gate("rzz", (0, 4), (0.9,)), C.Gate("cp", (1, 4), (1.1,))]
    c = C.Circuit(5, g)
    p = S.plan_json(5, g, S.SIM_C128, 0, S.default_options(flags=S.SIM_F_DIAG))
    phases = [op for op in p["ops"] if op["op"] == "phase"]
    assert len(phases) == 1
    assert p["stats"]["diag_fused"] == 4
    np.testing.assert_allclose(interpret(p), oracle.run(c), atol=1e-13)


def test_diagonal_detector_stops_at_stopped_qubit():
    # RZZ(0,1), H(1) [overlaps depSet -> uList, qubit 1 stopped], CP(1,2)
    # touches the stopped qubit -> must not be fused ahead of H(1)
    g = [C.Gate("rzz", (0, 1), (0.3,)), C.Gate("h", (1,)), C.Gate("cp", (1, 2), (0.7,)),
         C.Gate("rz", (0,), (0.2,))]
    c = C.Circuit(3, g)
    p = S.plan_json(3, g, S.SIM_C128, 0, S.default_options(flags=S.SIM_F_DIAG))
    kinds = [op["op"] for op in p["ops"]]
    assert kinds == ["phase", "gate", "phase"], kinds
    np.testing.assert_allclose(interpret(p), oracle.run(c), atol=1e-13)


def test_diagonal_detector_D_bound():
    g = [C.Gate("rzz", (i, i + 1), (0.1 * i,)) for i in range(8)]
    p = S.plan_json(12, g, S.SIM_C128, 0, S.default_options(flags=S.SIM_F_DIAG, max_diag_qubits=3))
    assert len([op for op in p["ops"] if op["op"] == "phase"]) == 4
    np.testing.assert_allclose(interpret(p), oracle.run(C.Circuit(12, g)), atol=1e-13)


def test_every_gate_emitted_once():
    c = C.diag_heavy(14, 300, 7)
    p = S.plan_json(c.n, c.gates, S.SIM_C128, 0, S.default_options(flags=S.SIM_F_DIAG))
    assert p["stats"]["gates_in"] == 314
    # ops + absorbed == inputs: nothing lost, nothing duplicated
    assert len(p["ops"]) + p["stats"]["diag_fused"] == 314


def test_invalid_gates_rejected():
    with pytest.raises(S.SimError) as e:
        S.plan_json(4, [C.Gate("cx", (1, 1))])
    assert e.value.code == S.SIM_EINVAL
    with pytest.raises(S.SimError):
        S.plan_json(4, [C.Gate("h", (4,))])
    with pytest.raises(S.SimError) as e:
        S.plan_json(35, [C.Gate("h", (0,))])
    assert e.value.code == S.SIM_EUNSUPPORTED


@pytest.mark.parametrize("maker", [lambda: C.layered(12, 6, 1), lambda: C.random_mixed(11, 120, 3, max_k=3),
                                   lambda: C.qft(10, 2), lambda: C.diag_heavy(12, 100, 4)])
def test_dense_block_plans_are_exact(maker):
    c = maker()
    opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG)
    p = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, opt)
    assert p["stats"]["dense_ops"] > 0
    assert all(op["op"] in ("gate", "phase") for op in p["ops"])
    assert all(len(op["qubits"]) == 5 for op in p["ops"] if op["op"] == "gate")
    np.testing.assert_allclose(interpret(p, basis=c.basis), oracle.run(c), atol=1e-12)


@pytest.mark.parametrize("maker", [lambda: C.layered(12, 6, 1), lambda: C.layered(16, 8, 2),
                                   lambda: C.random_mixed(14, 150, 3, max_k=3), lambda: C.qft(13, 2),
                                   lambda: C.diag_heavy(15, 120, 4)],
                         ids=["layered12", "layered16", "mixed14", "qft13", "diag15"])
def test_cache_blocked_dense_plans_are_exact(maker):
    """Complex64 split-TF32 blocks with cache blocking: runs of 5-qubit
    blocks share sweeps (dense_chunk ops) whose chunk holds qubits 0..3 and
    every block's qubits; the plan is exact and has no more sweeps than one
    sweep per block."""
    c = maker()
    base = S.SIM_F_TC | S.SIM_F_DIAG
    p = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, S.default_options(flags=base | S.SIM_F_BLOCK))
    sep = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, S.default_options(flags=base))
    chunks = [op for op in p["ops"] if op["op"] == "dense_chunk"]
    assert chunks and not any(op["op"] == "gate" and len(op["qubits"]) == 5 for op in p["ops"])
    for op in chunks:
        assert op["qin"][:4] == [0, 1, 2, 3] and op["qin"] == sorted(set(op["qin"])) and len(op["qin"]) == 12
        for blk in op["blocks"]:
            assert len(blk["qubits"]) == 5 and set(blk["qubits"]) <= set(op["qin"])
    # the blocked plan keeps the diagonal detector's output only when that is
    # cheaper, so its block count may differ from the one-sweep-per-block plan
    assert sum(len(op["blocks"]) for op in chunks) == p["stats"]["dense_ops"] <= sep["stats"]["dense_ops"] + 4
    assert p["stats"]["sweeps"] <= sep["stats"]["sweeps"]
    np.testing.assert_allclose(interpret(p, basis=c.basis), oracle.run(c), atol=1e-12)


def test_cache_blocked_dense_needs_a_full_chunk():
    """Below 12 qubits, complex128 states and the FP32 arm keep one sweep per
    block."""
    c = C.layered(11, 4, 1)
    opt = S.default_options(flags=S.SIM_F_TC | S.SIM_F_DIAG | S.SIM_F_BLOCK)
    assert not any(op["op"] == "dense_chunk" for op in S.plan_json(11, c.gates, S.SIM_C64, 0, opt)["ops"])
    c = C.layered(14, 4, 1)
    assert not any(op["op"] == "dense_chunk" for op in S.plan_json(14, c.gates, S.SIM_C128, 0, opt)["ops"])
    opt.dense_precision = S.SIM_DENSE_FP32
    assert not any(op["op"] == "dense_chunk" for op in S.plan_json(14, c.gates, S.SIM_C64, 0, opt)["ops"])


def test_swap_network_is_a_relabelling():
    """A qubit permutation given as SWAP gates (Eq. 4) costs no extra sweep
    per SWAP: the chunk stores apply it as a relabelling, a few sweeps for a
    full reversal, and the plan is exact."""
    for n in (14, 28):
        gates = [C.Gate("swap", (i, n - 1 - i)) for i in range(n // 2)]
        plan = S.plan_json(n, gates, S.SIM_C128, None)
        assert plan["stats"]["sweeps"] <= -(-n // 8) and plan["stats"]["gate_ops"] == 0
        if n == 14:
            rng = np.random.default_rng(3)
            a = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
            a /= np.linalg.norm(a)
            exp = oracle.run(C.Circuit(n, gates), state=a)
            np.testing.assert_allclose(interpret(plan, init_state=a), exp, atol=1e-12, rtol=0)


@pytest.mark.parametrize("name", ["layered", "qft", "mixed"])
def test_remap_plans_are_exact(name):
    """With qubit reordering through the block stores (SIM_F_REMAP) the
    frame changes between blocks and is restored at the end: still exact."""
    c = CIRCUITS[name](14)
    flags = S.SIM_F_DIAG | S.SIM_F_BOOST | S.SIM_F_BLOCK | S.SIM_F_FUSE | S.SIM_F_REMAP
    plan = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, S.default_options(flags=flags))
    np.testing.assert_allclose(interpret(plan, basis=c.basis), oracle.run(c), atol=1e-12, rtol=0)


def test_remap_cuts_sweeps_on_layered_circuits():
    """With 32 amplitudes per thread (the specialised kernels' shape) the
    qubit frame saves sweeps on the layered circuit (13 -> 11 at 28 qubits)."""
    c = C.layered(28, 20, 0)
    base = S.default_options(register_bits=5)
    rm = S.default_options(flags=base.flags | S.SIM_F_REMAP, register_bits=5)
    s0 = S.plan_json(c.n, c.gates, S.SIM_C64, 0, base)["stats"]["sweeps"]
    s1 = S.plan_json(c.n, c.gates, S.SIM_C64, 0, rm)["stats"]["sweeps"]
    assert s1 < s0


def test_euler_split_real_rotations_and_exact():
    """General one-qubit unitaries between diagonal gates are split into
    diag . real rotation . diag: the chunk sweeps on the full state carry only
    real 2x2 ops, the plan stays exact, and the phases do not add segments."""
    c = C.layered(14, 8, 3)
    plan = S.plan_json(c.n, c.gates, S.SIM_C128, c.basis, S.default_options())
    ops = [x for o in plan["ops"] if o["op"] == "chunk" and o["n"] == c.n for st in o["stages"] for x in st]
    dense = [x for x in ops if "dense" in x and len(x["dense"]) == 1]
    assert dense and all(abs(e[1]) == 0 for x in dense for e in x["matrix"])
    np.testing.assert_allclose(interpret(plan, basis=c.basis), oracle.run(c), atol=1e-12, rtol=0)
    # the leading phase of each rotation joins its layer's segment: at most
    # one phase segment per layer and register stage, not one per rotation
    nseg = sum(1 for x in ops if "phase" in x)
    assert nseg <= len(dense) // 4


@pytest.mark.parametrize("name,make,max_sweeps", [
    ("diag-heavy 28", lambda: C.diag_heavy(28, 500, 1), 7),
    ("qaoa 30", lambda: C.qaoa(30, 4, 3), 13),
    ("qft 30", lambda: C.qft(30, 2), 4),
    ("layered 30", lambda: C.layered(30, 20, 0), 15),
])
def test_benchmark_workloads_sweep_budget(name, make, max_sweeps):
    """The full-state passes of the benchmarked workloads, with the options
    the bench uses (defaults + specialised kernels): each sweep reads and
    writes the whole state, so a planner change that adds one shows up in
    every step.  The bounds are the counts the planner reaches now."""
    c = make()
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    st = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, opt)["stats"]
    assert st["sweeps"] <= max_sweeps, (name, st)
    assert st["chunk_ops"] + st["diag_ops"] >= 1


@pytest.mark.parametrize("name", ["mixed", "diagheavy", "qft", "qaoa", "layered"])
def test_plans_with_13_qubit_chunks_are_exact(name):
    """Chunks of 2^13 amplitudes (256 threads of 32 amplitudes, the shape
    the cost model picks for QAOA and layered circuits): plans at 15 qubits,
    run by the plan interpreter, equal the oracle's gate-by-gate state."""
    c = CIRCUITS[name](15 if name != "qaoa" else 14)
    opt = S.default_options(chunk_qubits=13, register_bits=5, flags=S.default_options().flags | S.SIM_F_JIT)
    plan = S.plan_json(c.n, c.gates, S.SIM_C64, c.basis, opt)
    assert any(o["op"] == "chunk" and o["C"] == 13 for o in plan["ops"])
    np.testing.assert_allclose(interpret(plan, basis=c.basis), oracle.run(c), atol=2e-7, rtol=0)


def test_chunk_shape_chosen_by_cost():
    """With no shape asked for, the specialised kernels' plans take 2^13-
    amplitude chunks only where they save enough sweeps (QAOA 30 q: 13 -> 9)
    and keep 2^12 where they do not (the 28-qubit diagonal-heavy stream)."""
    opt = S.default_options(flags=S.default_options().flags | S.SIM_F_JIT)
    q = C.qaoa(30, 4, 3)
    pq = S.plan_json(q.n, q.gates, S.SIM_C64, q.basis, opt)
    assert {o["C"] for o in pq["ops"] if o["op"] == "chunk" and o["n"] == 30} == {13}
    d = C.diag_heavy(28, 500, 1)
    pd = S.plan_json(d.n, d.gates, S.SIM_C64, d.basis, opt)
    assert {o["C"] for o in pd["ops"] if o["op"] == "chunk" and o["n"] == 28} == {12}
