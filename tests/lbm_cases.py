"""Shared helpers for the GPU parity tests: matched CUDA / oracle domains."""
import numpy as np

import oracle

XI, T19, W7, _, _ = oracle.lattice_tables()


def rel_err(gpu, ref, floor):
    """|g - o| / max(|o|, floor_q) per value (floor: w_q or t_q per row)."""
    g = np.asarray(gpu, dtype=np.float64)
    return np.abs(g - ref) / np.maximum(np.abs(ref), floor[:, None])


def pair(labels, affinity, periodic, **kw):
    import paper_2007_12266_gb300 as lbm
    dom = lbm.Domain(labels, affinity, periodic=periodic, **kw)
    okw = {k: v for k, v in kw.items() if k not in ("precision", "device")}
    ref = oracle.Oracle(labels, affinity, periodic, **okw)
    return dom, ref


def random_state(ref, seed, amp=0.05, phi_field=None):
    """A generic two-phase state near rest, exactly representable in fp32."""
    rng = np.random.default_rng(seed)
    N = ref.N
    if phi_field is None:
        phi = rng.uniform(-1, 1, N)
    else:
        phi = phi_field
    Ntot = 1.0 + 0.02 * rng.standard_normal(N)
    Na = 0.5 * Ntot * (1 + phi)
    Nb = 0.5 * Ntot * (1 - phi)
    f = T19[:, None] * (1 + amp * rng.standard_normal((19, N)))
    A = W7[:, None] * Na[None] * (1 + amp * rng.standard_normal((7, N)))
    B = W7[:, None] * Nb[None] * (1 + amp * rng.standard_normal((7, N)))
    return (f.astype(np.float32).astype(np.float64), A.astype(np.float32).astype(np.float64),
            B.astype(np.float32).astype(np.float64))


def set_both(dom, ref, state, step):
    """Load the same canonical state into both at the given step counter."""
    f, A, B = state
    ref.set_state(f, A, B, step=step)
    # the library places canonical values at the slots of its current parity;
    # a snapshot-like header carries the step count, so go through restore
    import struct
    N = ref.N
    header = struct.pack("<Qqqq", 0x4d50424c4c4f4332, N, step, 0)
    body = np.concatenate([f.astype(np.float32).ravel(), A.astype(np.float32).ravel(),
                           B.astype(np.float32).ravel()]).tobytes()
    dom.restore(header + body)


def compare_state(dom, ref):
    f, A, B = ref.state()
    return (rel_err(dom.distributions("f"), f, T19).max(),
            rel_err(dom.distributions("a"), A, W7).max(),
            rel_err(dom.distributions("b"), B, W7).max())
