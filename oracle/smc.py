"""Adaptive SMC / MLS^2MC sampler (oracle), FP64, step by step in the paper's order.

TEST INFRASTRUCTURE ONLY: part of the FP64 CPU oracle; never imported by the
product library.

Pieces and where they come from:
  cv, ESS                 Sec. 3.4, Eq. EQ:ESS:SMC_Update (population moments of
                          the unnormalised incremental weights)
  next increment          Sec. 3.4, Eqs. Eq_ESS_opt / Eq_cv_opt: the new inverse
                          temperature (or bridging temperature) is the argmin of
                          (cv - tau*)^2 over [min(beta+eps, 1), 1]
  ITU weights             Sec. 4.1: exp(-(beta_k - beta_{k-1}) Phi_l)
  LU / bridging weights   Sec. 3.2 and Sec. 4.1: exp(-beta (zeta_m - zeta_{m-1}) (Phi_l - Phi_{l-1}))
  evidence                Sec. 5.1.3: the product of the mean incremental weights
  resampling              Sec. 2.4 (resample before the Markov move); the scheme
                          (systematic) is not fixed by the paper
  Markov kernel           Sec. 5 uses one random-walk Metropolis step; here the
                          preconditioned Crank-Nicolson proposal the paper names as
                          the better choice in high dimension (Cotter et al. 2013),
                          that random walk, and (not in the paper) a random walk
                          whose covariance is the particle population's
  update scheme           Sec. 4.4, Eq. eq_updatescheme_final with the cv^LU
                          predictor on J~ particles (Sec. 4.4)
"""
import math

import numpy as np

from . import philox


def cv(w):
    """Coefficient of variation StD/E of unnormalised weights, population (1/J) moments."""
    w = np.asarray(w, dtype=np.float64)
    m = np.mean(w)
    return math.sqrt(max(np.mean(w * w) - m * m, 0.0)) / m


def ess(w):
    return w.size / (1.0 + cv(w) ** 2)


def cv_of_increment(a, delta):
    """cv of w_j = exp(-delta * a_j); shifting a by its minimum leaves cv unchanged."""
    a = np.asarray(a, dtype=np.float64)
    return cv(np.exp(-delta * (a - a.min())))


def next_increment(a, dmax, tau, eps, iters=100):
    """argmin over delta in [min(eps, dmax), dmax] of (cv(exp(-delta a)) - tau)^2.

    cv(delta) is non-decreasing in delta, so the argmin is the root of
    cv = tau when it lies inside the interval, else the nearer endpoint. The root
    is found by a fixed number of bisection halvings. When cv(dmax) <= tau
    (this includes all a equal, where cv == 0) the whole remaining step is taken.
    """
    dmin = min(eps, dmax)
    if cv_of_increment(a, dmax) <= tau:
        return dmax
    if cv_of_increment(a, dmin) >= tau:
        return dmin
    lo, hi = dmin, dmax
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if cv_of_increment(a, mid) > tau:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def log_mean_weight(a, delta):
    """log( (1/J) sum_j exp(-delta a_j) ), evaluated stably (log-sum-exp)."""
    a = np.asarray(a, dtype=np.float64)
    amin = a.min()
    return -delta * amin + math.log(np.mean(np.exp(-delta * (a - amin))))


def systematic_resample(logw, U):
    """Ancestor indices: a(i) = min{ j : c_j > (U + i)/J }, c the normalised-weight cumsum, c_{J-1} = 1."""
    logw = np.asarray(logw, dtype=np.float64)
    J = logw.size
    w = np.exp(logw - logw.max())
    c = np.cumsum(w / w.sum())
    c[-1] = 1.0
    pos = (U + np.arange(J)) / J
    return np.searchsorted(c, pos, side='right')


def pcn_propose(theta, xi, s):
    """theta' = sqrt(1 - s^2) theta + s xi (prior-reversible for N(0, I))."""
    return math.sqrt(1.0 - s * s) * theta + s * xi


def rwm_propose(theta, xi, s):
    """theta' = theta + s xi: the Gaussian random walk of Sec. 5 (proposal covariance s^2 I,
    s^2 = 2.38^2 / N_sto in the paper)."""
    return theta + s * xi


def population_chol(theta, ridge=1e-4):
    """Lower Cholesky factor L of the covariance-shaped random walk's proposal covariance (not in
    the paper, whose random walk has covariance s^2 I): the covariance of the particle population,
    C = (1/J) sum_j (theta_j - mean)(theta_j - mean)^T, plus ridge * (tr C / K + 1e-12) I, which
    keeps it positive definite when the population spans fewer than K directions (the 1e-12, far
    below any spread of a prior N(0, I) sample, covers a population of identical particles, whose C
    is rounding noise). It is formed from the population before an update's moves, so every move of
    the update uses the same symmetric proposal and leaves the update's target invariant."""
    J, K = theta.shape
    d = theta - theta.mean(axis=0)
    C = d.T @ d / J
    C = C + ridge * (np.trace(C) / K + 1e-12) * np.eye(K)
    return np.linalg.cholesky(C)


def rwm_cov_propose(theta, xi, s, L):
    """theta' = theta + s L xi for every row (the covariance-shaped random walk)."""
    return theta + s * (xi @ L.T)


def log_prior_ratio(theta_new, theta):
    """log mu0(theta') - log mu0(theta) for mu0 = N(0, I), one value per row."""
    return -0.5 * (np.sum(theta_new * theta_new, axis=1) - np.sum(theta * theta, axis=1))


class Sampler:
    """MLS^2MC (Sec. 4) on a hierarchy of levels; single-level SMC when there is one level.

    evaluate(level, theta) -> Phi must return the potential on that level for each
    row of theta. Randomness comes from Philox4x32-10 with the library's draw layout,
    so with the same seed the oracle and the GPU sampler consume identical numbers.
    """

    def __init__(self, evaluate, n_levels, K, J, J_tilde=100, n_mcmc=5, tau_star=1.0,
                 tau_lu=None, eps=1e-6, s_pcn=0.2, seed=0, theta0=None, proposal="pcn", tau_min=0.0,
                 accept_target=0.0):
        self.evaluate_raw = evaluate
        self.L = n_levels
        self.K = K
        self.J = J
        self.J_tilde = min(J_tilde, J)
        self.n_mcmc = n_mcmc
        self.tau = tau_star
        self.tau_lu = tau_star if tau_lu is None else tau_lu
        self.eps = eps
        self.s = s_pcn
        if proposal not in ("pcn", "rwm", "rwm_cov"):
            raise ValueError("proposal must be 'pcn', 'rwm' or 'rwm_cov'")
        self.proposal = proposal
        self.tau_min = tau_min         # > 0: the scheme u' of Sec. 4.5 (adaptive maximum level)
        # > 0: the Markov kernel's step adapts between updates, s <- s exp(a - accept_target) with a
        # the last update's acceptance rate (clamped to [1e-4, 1] for pCN, [1e-4, 100] for the random
        # walk); an update's step depends on finished updates only, so its kernel leaves its target
        # invariant (the paper fixes the step)
        self.accept_target = accept_target
        self.step_size = s_pcn
        self.last_unique = J
        self.terminated = False
        self.seed = seed
        self.evals = np.zeros(n_levels, dtype=np.int64)
        self.level = 0
        self.beta = 0.0
        self.prev_lu = True            # u(-1) = (0, 0), u(0) = (0, 1): the first update is an ITU
        self.log_z = 0.0
        self.stage = 0                 # one per importance-sampling update (ITU or bridging step)
        self.mcmc_event = 0
        self.path = []                 # one record per update
        self.accepts = []
        if theta0 is None:
            theta0 = philox.normals(J, K, 0, philox.PURPOSE_PRIOR, seed)
        self.theta = np.array(theta0, dtype=np.float64)
        self.phi = self.evaluate(0, self.theta)

    def evaluate(self, level, theta):
        self.evals[level] += theta.shape[0]
        return np.asarray(self.evaluate_raw(level, theta), dtype=np.float64)

    @property
    def done(self):
        return self.beta >= 1.0 and (self.level == self.L - 1 or self.terminated)

    # -- importance sampling + resampling ---------------------------------------------------
    def _reweight_resample(self, a, dmax):
        delta = next_increment(a, dmax, self.tau, self.eps)
        self.log_z += log_mean_weight(a, delta)
        U = philox.uniform_scalar(self.stage, philox.PURPOSE_RESAMPLE, self.seed)
        anc = systematic_resample(-delta * a, U)
        self.last_unique = int(np.unique(anc).size)
        w = np.exp(-delta * (a - a.min()))
        return delta, anc, cv(w)

    def _mcmc(self, target):
        """n_mcmc pCN (or random-walk) Metropolis steps; target(theta) -> (Phi_target, caches)
        evaluates the proposal."""
        acc = 0
        phi_t, caches = target(None)
        s = self.step_size if self.accept_target > 0.0 else self.s
        self.last_step = s
        # the covariance-shaped walk takes its covariance from the population before the moves
        L = population_chol(self.theta) if self.proposal == "rwm_cov" else None
        for _ in range(self.n_mcmc):
            xi = philox.normals(self.J, self.K, self.mcmc_event, philox.PURPOSE_PCN_XI, self.seed)
            u = philox.uniforms_open(self.J, self.mcmc_event, philox.PURPOSE_PCN_U, self.seed)
            if self.proposal == "pcn":
                prop = pcn_propose(self.theta, xi, s)
                phi_t_new, caches_new = target(prop)
                ok = np.log(u) < -(phi_t_new - phi_t)
            else:   # random walks: the prior ratio enters the acceptance
                prop = rwm_propose(self.theta, xi, s) if L is None else rwm_cov_propose(self.theta, xi, s, L)
                phi_t_new, caches_new = target(prop)
                ok = np.log(u) < -(phi_t_new - phi_t) + log_prior_ratio(prop, self.theta)
            self.theta[ok] = prop[ok]
            phi_t = np.where(ok, phi_t_new, phi_t)
            for c, cn in zip(caches, caches_new):
                c[ok] = cn[ok]
            acc += int(ok.sum())
            self.mcmc_event += 1
        rate = acc / (self.n_mcmc * self.J) if self.n_mcmc > 0 else 0.0
        if self.accept_target > 0.0:
            hi = 1.0 if self.proposal == "pcn" else 100.0
            self.step_size = min(hi, max(1e-4, self.step_size * math.exp(rate - self.accept_target)))
        return rate

    # -- the two update types ----------------------------------------------------------------
    def _itu(self):
        l = self.level
        delta, anc, cvw = self._reweight_resample(self.phi, 1.0 - self.beta)
        self.theta = self.theta[anc]
        self.phi = self.phi[anc]
        self.beta = 1.0 if delta >= 1.0 - self.beta else self.beta + delta
        beta = self.beta

        def target(prop):
            if prop is None:
                return beta * self.phi, [self.phi]
            p = self.evaluate(l, prop)
            return beta * p, [p]
        rate = self._mcmc(target)
        self.path.append(dict(kind='ITU', level=l, beta=self.beta, zeta=None, delta=delta,
                              cv=cvw, accept=rate, n_unique=self.last_unique, step=self.last_step))
        self.stage += 1
        self.prev_lu = False

    def _lu(self, phi_fine_head):
        l = self.level
        rest = self.evaluate(l + 1, self.theta[phi_fine_head.size:])
        phi_f = np.concatenate([phi_fine_head, rest])
        phi_c = self.phi
        zeta = 0.0
        beta = self.beta
        nb = 0
        while zeta < 1.0:
            a = beta * (phi_f - phi_c)
            delta, anc, cvw = self._reweight_resample(a, 1.0 - zeta)
            self.theta = self.theta[anc]
            phi_f = phi_f[anc]
            phi_c = phi_c[anc]
            zeta = 1.0 if delta >= 1.0 - zeta else zeta + delta
            z = zeta

            def target(prop, z=z):
                if prop is None:
                    return beta * ((1.0 - z) * phi_c + z * phi_f), [phi_c, phi_f]
                pc = self.evaluate(l, prop)
                pf = self.evaluate(l + 1, prop)
                return beta * ((1.0 - z) * pc + z * pf), [pc, pf]
            rate = self._mcmc(target)
            nb += 1
            self.path.append(dict(kind='LU', level=l + 1, beta=beta, zeta=zeta, delta=delta,
                                  cv=cvw, accept=rate, n_unique=self.last_unique, step=self.last_step))
            self.stage += 1
        self.level = l + 1
        self.phi = phi_f
        self.prev_lu = True
        return nb

    def step(self):
        """One update of Eq. eq_updatescheme_final (or eq_updatescheme_final_Lmax when tau_min > 0):
        an ITU, or a whole LU with its bridging steps; None when the sampler stops."""
        if self.done:
            return None
        l = self.level
        if l == self.L - 1:
            self._itu()
        elif self.beta >= 1.0:
            # beta = 1: an ITU is impossible, so the level is raised. Under u' (Sec. 4.5) the
            # information gain of that level update is assessed first by cv^LU on the first J~
            # particles: below tau_min the sampler stops on this level (no update is recorded).
            if self.tau_min > 0.0:
                jt = self.J_tilde
                head = self.evaluate(l + 1, self.theta[:jt])
                d = head - self.phi[:jt]
                cv_lu = cv(np.exp(-self.beta * (d - d.min())))
                if cv_lu < self.tau_min:
                    self.terminated = True
                    return None
                self._lu(head)
            else:
                self._lu(np.empty(0))
        elif self.prev_lu:
            self._itu()
        else:
            jt = self.J_tilde
            head = self.evaluate(l + 1, self.theta[:jt])
            cv_lu = cv(np.exp(-self.beta * ((head - self.phi[:jt]) - (head - self.phi[:jt]).min())))
            if cv_lu < self.tau_lu:
                self._itu()
                self.path[-1]['cv_lu'] = cv_lu
            else:
                self._lu(head)
        return self.path[-1]

    def run(self, max_updates=10000):
        while not self.done and len(self.path) < max_updates:
            self.step()
        return self

    def moments(self):
        return self.theta.mean(axis=0), self.theta.var(axis=0)
