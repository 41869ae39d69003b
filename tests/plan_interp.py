"""Numpy interpreter of the optimizer's JSON plan (test helper).

Applies each planned operation to a complex128 state exactly as its
definition says -- a dense matrix on listed qubits, a phase polynomial
exp(2 pi i sum_t w_t prod_{j in mask_t} x_j / 2^64), the store permutation of
a cached chunk, a tensor product of sub-states -- so that a test can compare
``interpret(plan)`` with the oracle and check that the optimizer's rewriting
(fusion, diagonal detection, reordering, relabelling, boosting) is exact.
"""
import numpy as np


def apply_matrix(a, n, pos, M):
    k = len(pos)
    t = a.reshape([2] * n)
    Mt = np.asarray(M).reshape([2] * (2 * k))
    # matrix axes: (r_{k-1}..r_0, c_{k-1}..c_0); state axis of qubit q is n-1-q
    col_axes = list(range(k, 2 * k))
    st_axes = [n - 1 - pos[k - 1 - i] for i in range(k)]
    out = np.tensordot(Mt, t, axes=(col_axes, st_axes))
    # out axes: r_{k-1}..r_0 then the remaining state axes in order
    rest = [ax for ax in range(n) if ax not in st_axes]
    cur = st_axes + rest
    inv = np.argsort(cur)
    return np.transpose(out, inv).reshape(-1)


def phase_factors(n, terms, wbits=64):
    x = np.arange(1 << n, dtype=np.uint64)
    w = np.zeros(1 << n, dtype=np.uint64)
    for m, wt in terms:
        m = np.uint64(int(m))
        wt = int(wt)
        if wbits == 32:   # the complex64 kernels round every term to 32 bits
            wt = ((wt + (1 << 31)) >> 32) << 32
            wt &= (1 << 64) - 1
        w += np.where((x & m) == m, np.uint64(wt), np.uint64(0))
    ang = w.astype(np.int64).astype(np.float64) * (2 * np.pi / 2.0 ** 64)
    return np.exp(1j * ang)


def permute(a, n, qin, qout):
    x = np.arange(1 << n, dtype=np.uint64)
    qmask = 0
    for q in qin:
        qmask |= 1 << q
    y = x & np.uint64(((1 << n) - 1) & ~qmask)
    for i, qi in enumerate(qin):
        y |= ((x >> np.uint64(qi)) & np.uint64(1)) << np.uint64(qout[i])
    out = np.empty_like(a)
    out[y] = a
    return out


def _matrix(js):
    return np.array([complex(r, i) for r, i in js])


def interpret(plan, init_state=None, basis=0):
    n = plan["n"]
    wbits = plan["wbits"]
    bufs = {}
    for b, nq in enumerate(plan["buffers"]):
        bufs[b] = np.zeros(1 << nq, complex)
    if init_state is not None:
        bufs[0] = np.array(init_state, complex)
    else:
        bufs[0][basis] = 1.0
    for op in plan["ops"]:
        kind = op["op"]
        b, nb = op["buf"], op["n"]
        a = bufs[b]
        if kind == "init":
            a = np.zeros(1 << nb, complex)
            a[int(op["basis"])] = 1.0
        elif kind == "gate":
            q = op["qubits"]
            dim = 1 << len(q)
            a = apply_matrix(a, nb, q, _matrix(op["matrix"]).reshape(dim, dim))
        elif kind == "phase":
            a = a * phase_factors(nb, op["terms"], wbits)
        elif kind == "chunk":
            for st in op["stages"]:
                for x in st:
                    if "dense" in x:
                        q = x["dense"]
                        dim = 1 << len(q)
                        a = apply_matrix(a, nb, q, _matrix(x["matrix"]).reshape(dim, dim))
                    else:
                        a = a * phase_factors(nb, x["phase"], wbits)
            a = permute(a, nb, op["qin"], op["qout"])
        elif kind == "dense_chunk":
            # a cache-blocked sweep of dense blocks: each block is a matrix on
            # its qubits, applied in order (the chunk changes no labels)
            for blk in op["blocks"]:
                q = blk["qubits"]
                dim = 1 << len(q)
                a = apply_matrix(a, nb, q, _matrix(blk["matrix"]).reshape(dim, dim))
        elif kind == "tensor":
            a = np.kron(bufs[op["hi"]], bufs[op["lo"]])
        else:
            raise ValueError(kind)
        bufs[b] = a
    return bufs[0]
