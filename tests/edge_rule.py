"""The per-edge precision rule of the MBH_MIXED heterodyne, restated for the GPU tests (host
side, from a prepared reference's summary data)."""
import numpy as np


def f32_edge_count(ref, g, kappa=None, budget=3e-4, eps32=3e-7, delta_max=3.0, group=4, rtol=1e-9):
    """The per-edge precision rule of MBH_MIXED recomputed from the reference's summary data:
    each edge meets the summary data of the bin above it (as its lower edge) and below it (as
    its upper edge), with the per-bin linear interpolation of r (Eqs. 14 and 17) giving five
    weights per channel, for <d|h> w_ar Re delta + w_ai Im delta and for <h|h> w_br Re delta +
    w_q |delta|^2 + w_c Re(delta_prev conj delta); its sensitivity bounds |d lnL / d delta| for
    |delta| and its neighbours' <= delta_max, S_e = 4 sum_c (|w_ar| + |w_ai| + |w_br|/2 +
    delta_max |w_q| + delta_max (|w_c| + |w_cn|)/2) with w_cn the next edge's w_c, times kappa_e
    (higher modes: the error growth where the reference's modes cancel; 1 by default).  Edges
    are taken in aligned groups of `group`, the groups of smallest summed sensitivity first,
    while eps32 times the sum stays within budget.  Returns the edge counts at budget (1 -/+
    rtol): the rule's count lies between them."""
    r = ref.read()
    q, edges = r["summary"], r["edges"]
    fe = g["f0"] + edges * g["df"]
    iw = 1.0 / (fe[1:] - fe[:-1])
    E = len(edges) - 1
    S = np.zeros(E + 1)
    for c in range(3):
        a0r, a0i, a1r, a1i, b0, b1 = (q[:, c, j] for j in range(6))
        war, wai, wbr, wq, wc = (np.zeros(E + 1) for _ in range(5))
        war[:-1] += 0.5 * a0r - a1r * iw
        war[1:] += 0.5 * a0r + a1r * iw
        wai[:-1] += 0.5 * a0i - a1i * iw
        wai[1:] += 0.5 * a0i + a1i * iw
        wbr[:-1] += b0 - 2 * b1 * iw
        wbr[1:] += b0 + 2 * b1 * iw
        wq[:-1] += 0.25 * b0 - b1 * iw
        wq[1:] += 0.25 * b0 + b1 * iw
        wc[1:] = 0.5 * b0
        wcn = np.zeros(E + 1)   # the next edge's cross term with this one
        wcn[:-1] = 0.5 * b0
        S += 4 * (np.abs(war) + np.abs(wai) + 0.5 * np.abs(wbr) + delta_max * np.abs(wq)
                  + 0.5 * delta_max * (np.abs(wc) + np.abs(wcn)))
    if kappa is not None:
        S = S * kappa
    ng = (E + 1 + group - 1) // group
    gs = np.array([S[i * group:(i + 1) * group].sum() for i in range(ng)])
    size = np.array([min(E + 1, (i + 1) * group) - i * group for i in range(ng)])
    order = np.argsort(gs, kind="stable")
    cum = np.cumsum(gs[order]) * eps32

    def count(b):
        return int(size[order][cum <= b].sum())
    return count(budget * (1 - rtol)), count(budget * (1 + rtol))
