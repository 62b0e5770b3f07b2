"""FP64 reference of the inverse-design loop that drives the forward and gradient solves.

TEST INFRASTRUCTURE ONLY: imported by tests/ and never by the product path; it shares no code with
the CUDA library (the gradient comes from the FP64 oracle in oracle.py).

arXiv 2412.12360 Sec. 3.2-3.3 optimises device designs with gradients from the time-reversal solve,
the design quantised to two materials. The reading built here (the paper names neither its
parameterisation nor its optimiser in detail):
  - densities rho in [0, 1] on the design box, eps = eps_lo + (eps_hi - eps_lo) rho;
  - binarisation by the smoothed Heaviside projection rho = P_beta(theta) of latent variables theta
    (Wang, Lazarov and Sigmund, Struct. Multidisc. Optim. 43, 2011), beta raised over the iterations;
  - Adam (Kingma and Ba, ICLR 2015) on theta, clamped to [0, 1].
Each function below writes its formula out as stated there, in float64.
"""
import numpy as np

from . import oracle as O


def projection(theta, beta, eta=0.5):
    """P(theta) = (tanh(beta eta) + tanh(beta (theta - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)));
    beta = 0 is the identity (the beta -> 0 limit)."""
    theta = np.asarray(theta, dtype=np.float64)
    if beta == 0:
        return theta.copy()
    num = np.tanh(beta * eta) + np.tanh(beta * (theta - eta))
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return num / den


def projection_grad(theta, beta, eta=0.5):
    """dP/dtheta = beta (1 - tanh^2(beta (theta - eta))) / (tanh(beta eta) + tanh(beta (1 - eta)))."""
    theta = np.asarray(theta, dtype=np.float64)
    if beta == 0:
        return np.ones_like(theta)
    den = np.tanh(beta * eta) + np.tanh(beta * (1.0 - eta))
    return beta * (1.0 - np.tanh(beta * (theta - eta)) ** 2) / den


def adam_step(theta, m, v, g_rho, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, proj_beta=0.0, proj_eta=0.5):
    """One Adam step on theta for the loss gradient dL/drho at rho = P(theta); returns the new
    (theta, m, v, rho) with theta clamped to [0, 1] and rho = P(theta_new)."""
    g = np.asarray(g_rho, dtype=np.float64) * projection_grad(theta, proj_beta, proj_eta)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    theta = np.clip(np.asarray(theta, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), 0.0, 1.0)
    return theta, m, v, projection(theta, proj_beta, proj_eta)


def set_density(scene, rho, eps_lo, eps_hi):
    """Write eps_inv = 1 / (eps_lo + (eps_hi - eps_lo) rho) into the scene's design box."""
    lo, hi = scene.design_lo, scene.design_hi
    eps = eps_lo + (eps_hi - eps_lo) * np.asarray(rho, dtype=np.float64)
    scene.eps_inv[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = 1.0 / eps


def design_loop(scene, nsteps, theta0, iters, objective, lr, eps_lo, eps_hi, beta_of=lambda it: 0.0,
                proj_eta=0.5, beta1=0.9, beta2=0.999, eps=1e-8):
    """Run `iters` design iterations; objective(det) -> (L, dL/ddet). Returns (losses, theta)."""
    theta = np.asarray(theta0, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for it in range(iters):
        beta = beta_of(it)
        rho = projection(theta, beta, proj_eta)
        set_density(scene, rho, eps_lo, eps_hi)
        det = O.forward(scene, nsteps)[1]
        L, dL_ddet = objective(det)
        losses.append(float(L))
        dL_deps = O.gradient(scene, nsteps, dL_ddet, O.METHOD_TIME_REVERSAL)[0]
        g_rho = dL_deps * (eps_hi - eps_lo)
        theta, m, v, _ = adam_step(theta, m, v, g_rho, it + 1, lr, beta1, beta2, eps, beta, proj_eta)
    return losses, theta
