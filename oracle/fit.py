"""Oracle (test infrastructure only): the table-fitting loop in float64.

Loss per query (the fit workload's reading; the paper has no fitting): L_q = w_v (R - R_t)^2 +
w_n |n - n_t|^2 on the query outputs of query.c; its gradient with respect to the stored records
comes from the reverse mode in adjoint.c with upstream dL/dR = 2 w_v (R - R_t), dL/dn = 2 w_n (n - n_t).
Adam as defined by Kingma & Ba (ICLR 2015), Algorithm 1, with bias correction.
"""
import numpy as np

from . import query, query_vjp


def loss_and_grad(pool, off, Ns, dirs, R_t, n_t, w_value=1.0, w_normal=1.0, glyph=None, r0=None):
    out = query(pool, off, Ns, dirs, glyph=glyph, r0=r0)
    eR = out["R"] - R_t
    en = out["normal"] - n_t
    loss = float(w_value * (eR ** 2).sum() + w_normal * (en ** 2).sum())
    dpool, _ = query_vjp(pool, off, Ns, dirs, gR=2.0 * w_value * eR, gn=2.0 * w_normal * en, glyph=glyph, r0=r0,
                         want_ddirs=False)
    return loss, dpool


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of float64 arrays (returns new p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
