"""The overlap of consecutive kernels on the two-kernel path, as a schedule
model (no GPU): which phases of which kernels may run at the same time, and
what each phase reads and writes.

Rules (snn_kernels.cu, snn_host.cpp capture_steps): every kernel triggers its
dependent right after its own griddepcontrol.wait, so a kernel launched with
programmatic serialization can overlap only the part after the wait of the
kernel directly before it.  A delivery pass always follows its update that
way; an update follows a pass that way; an update that follows an update
starts after it.  The input of step t is buffer t mod 2 kmin, the spike list
of step t is slot t mod (n_delay + kmin).  Concurrent phases must not touch
the same buffer or slot unless both only add to it (order-free int32 sums).
"""
import pytest


def _phases(t, kmin, n_delay):
    """(kernel, phase) -> list of (resource, index, mode) for the update of
    step t and, after the last step of an exchange period, its pass."""
    nbuf, D = 2 * kmin, n_delay + kmin
    out = []
    u_pre = [("state", 0, "r")]
    u_post = [("acc", t % nbuf, "r"), ("acc", t % nbuf, "w"), ("state", 0, "w"),
              ("hist", t % D, "add"), ("cnt", t % D, "add")]
    out.append((("U", t), u_pre, u_post))
    if (t + 1) % kmin == 0:
        d_pre, d_post = [], []
        for j in range(kmin):
            T = t + 1 + j
            for d in range(kmin, n_delay + 1):
                src = T - d
                if src == t:
                    continue            # the step's own spikes: after the wait
                if src >= 0:
                    d_pre += [("hist", src % D, "r"), ("cnt", src % D, "r")]
            d_pre.append(("acc", T % nbuf, "add"))
        d_post += [("hist", t % D, "r"), ("cnt", t % D, "r"), ("acc", (t + kmin) % nbuf, "add")]
        d_post += [("cnt", (t + 1 + i) % D, "w") for i in range(kmin)]
        out.append((("D", t), d_pre, d_post))
    return out


def _conflict(a, b):
    for ra, ia, ma in a:
        for rb, ib, mb in b:
            if ra != rb or ia != ib:
                continue
            if ma == "add" and mb == "add":
                continue                # order-free sums
            if ma == "r" and mb == "r":
                continue
            return (ra, ia, ma, mb)
    return None


@pytest.mark.parametrize("kmin,n_delay", [(1, 1), (1, 20), (1, 254), (2, 7), (4, 7), (10, 20), (20, 20),
                                          (3, 30), (7, 8)])
def test_overlapping_phases_touch_disjoint_buffers_and_slots(kmin, n_delay):
    seq = []
    for t in range(0, 6 * max(kmin, 1) + 3 * n_delay):
        seq += _phases(t, kmin, n_delay)
    for i in range(1, len(seq)):
        (prev, _, prev_post), (cur, cur_pre, _) = seq[i - 1], seq[i]
        overlapped = cur[0] == "D" or prev[0] == "D"   # a pass after its update, an update after a pass
        if not overlapped:
            continue
        c = _conflict(prev_post, cur_pre)
        assert c is None, (kmin, n_delay, prev, cur, c)


def test_one_buffer_per_step_of_the_period_would_clash():
    """kmin + 1 input buffers would do (the pass writes t + 1 .. t + kmin, the
    update reads t); 2 kmin are kept so that windows starting at the same step
    mod 2 kmin share a captured graph.  kmin buffers would let the pass after
    step t add into the buffer the update of step t is reading and clearing."""
    for kmin in (1, 2, 4, 10):
        ends = [t for t in range(5 * kmin) if (t + 1) % kmin == 0]
        assert any(t % kmin in {(t + 1 + j) % kmin for j in range(kmin)} for t in ends)
        for nbuf in (kmin + 1, 2 * kmin):
            assert not any(t % nbuf in {(t + 1 + j) % nbuf for j in range(kmin)} for t in ends)
