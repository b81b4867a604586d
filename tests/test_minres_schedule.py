"""The fused MINRES step's schedule, restated in numpy and checked against
SciPy's MINRES (no GPU, no oracle).

The fused step (the n1 pass with the Lanczos step folded in) keeps the
Lanczos vectors unnormalised (u_k = beta_k v_k) in three rotating buffers
(u_k in buffer k mod 3), the w vectors in two (w_j by the parity of j),
applies the w update one iteration late, and adds tau_j w_j to x for three
j at once on every third iteration; the flush after the loop adds what is
pending.  This test runs that schedule, with the scalar recurrences of the
Givens step (Paige and Saunders' MINRES), on small symmetric systems and
compares the iterate after each number of iterations with SciPy's.
"""
import numpy as np
import pytest

scipy_linalg = pytest.importorskip("scipy.sparse.linalg")


def fused_schedule(A, b, iters, deferred=True):
    n = b.size
    beta1 = np.linalg.norm(b)
    st = dict(beta=beta1, beta_prev=0.0, alpha=0.0, c=-1.0, s=0.0, dbar=0.0, eps=0.0, phibar=beta1,
              d=0.0, e=0.0, ig=0.0, tau=0.0, ib=0.0, t1=0.0, t2=0.0, k=0)
    u = [np.zeros(n), b.copy(), np.zeros(n)]          # u_0, u_1, (u_2)
    w = [np.zeros(n), np.zeros(n)]                     # w by parity
    x = np.zeros(n)

    def givens(bn2):
        beta_next = np.sqrt(max(bn2, 0.0))
        alpha, c, s, dbar = st["alpha"], st["c"], st["s"], st["dbar"]
        delta = c * dbar + s * alpha
        gbar = s * dbar - c * alpha
        eps_next = s * beta_next
        dbar_next = -c * beta_next
        gamma = np.hypot(gbar, beta_next) or 1e-300
        cn, sn = gbar / gamma, beta_next / gamma
        tau = cn * st["phibar"]
        st.update(d=delta, e=st["eps"], ig=1.0 / gamma, t2=st["t1"], t1=st["tau"], tau=tau,
                  ib=1.0 / st["beta"], c=cn, s=sn, dbar=dbar_next, eps=eps_next, phibar=sn * st["phibar"],
                  beta_prev=st["beta"], beta=beta_next, k=st["k"] + 1)

    for _ in range(iters):
        k = st["k"]
        uk, um, un = u[(k + 1) % 3], u[k % 3], (k + 2) % 3
        p = A @ uk
        st["alpha"] = (uk @ p) / st["beta"] ** 2                     # the n3 pass's energy
        cv = -st["beta"] / st["beta_prev"] if st["beta_prev"] > 0 else 0.0
        unew = p / st["beta"] - (st["alpha"] / st["beta"]) * uk + cv * um
        if k > 0:                                                      # lagged update: w_k
            wa, wb = w[(k - 1) % 2], w[k % 2]                           # w_{k-1}, w_{k-2}
            wn = (um * st["ib"] - st["d"] * wa - st["e"] * wb) * st["ig"]
            if not deferred:
                x += st["tau"] * wn
            elif k % 3 == 0:
                x += st["t2"] * wb + st["t1"] * wa + st["tau"] * wn
            w[k % 2] = wn
        u[un] = unew
        givens(unew @ unew)
    # flush: w_K, and the pending tau_j w_j
    K = st["k"]
    if K > 0:
        wa, wb = w[(K - 1) % 2], w[K % 2]
        wn = (u[K % 3] * st["ib"] - st["d"] * wa - st["e"] * wb) * st["ig"]
        r = (K - 1) % 3 if deferred else 0
        x = x + (st["t2"] * wb if r == 2 else 0) + (st["t1"] * wa if r >= 1 else 0) + st["tau"] * wn
    return x, st["phibar"] / beta1


def scipy_minres(A, b, iters):
    out = []
    scipy_linalg.minres(A, b, rtol=0.0, maxiter=iters, callback=lambda xk: out.append(xk.copy()))
    return out[-1]


@pytest.mark.parametrize("n,seed,indefinite", [(30, 0, False), (41, 1, False), (36, 2, True)])
@pytest.mark.parametrize("iters", [1, 2, 3, 4, 5, 6, 7, 11, 12, 13])
def test_fused_schedule_matches_scipy_minres(n, seed, indefinite, iters):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = rng.uniform(0.5, 4.0, n)
    if indefinite:
        ev[: n // 3] *= -1.0
    A = (Q * ev) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    ref = scipy_minres(A, b, iters)
    for deferred in (False, True):
        x, _ = fused_schedule(A, b, iters, deferred)
        assert np.linalg.norm(x - ref) <= 1e-10 * np.linalg.norm(ref), (deferred, iters)

