"""Oracle: the hydrogen ground-state iteration of Sec. 6.2 (eq. Kalos),
phi = -2 G_mu V phi with V = -1/r, mu = sqrt(-2E).

Test infrastructure only (see ``oracle/__init__``).

Units.  The library's functions live on the unit cube; a physical cube of
side L (atomic units) maps to it by x = L u, with the nucleus at u0.  For
f~(u) = f(L u):  V~(u) = -1 / (L |u - u0|) (a point charge -1/L at u0), and
G_mu f (L u) = L^2 (G~_{mu L} f~)(u), where G~_{nu} is the convolution with
e^{-nu r} / (4 pi r) on the unit cube (K_{nu,1}, the library's operator with
alpha = 1).  L2 norms carry a factor L^{3/2}; energies are ratios of inner
products, in which L^3 cancels.

Steps (Sec. 6.2), one call of ``kalos_step``:
  2. P = V phi (``product.multiply``, a point charge);
  3. phi_new = -2 G_mu P (compress, Algorithm 3, eq. g_assemble, x -2 L^2);
  4. E_new from phi_new.  The paper's energy uses <grad phi_new, grad phi_new>;
     reading used here: that term is taken from the equation phi_new solves,
     (-Laplacian + mu^2) phi_new = -2 V phi, by integration by parts:
       (1/2) <grad phi_new, grad phi_new> = -<V phi, phi_new> - (mu^2/2) ||phi_new||^2,
     so E_new = (-<V phi, phi_new> - (mu^2/2) ||phi_new||^2
                 + <V phi_new, phi_new>) / ||phi_new||^2
     and no derivative operator is needed.
  5. mu = sqrt(-2 E_new), phi = phi_new / ||phi_new||.
The skeleton stays that of the starting tree (reading: the paper re-adapts
its trees with the products of [A-B-G-V:2002], which it does not describe).

Parity pin (tests/test_oracle_product.py): started from the exact ground
state e^{-r} / sqrt(pi) with mu = 1, one step returns E_new close to -1/2 and
phi_new close to phi; and from e^{-zeta r} the energy estimate moves toward
-1/2.
"""
import math

from . import apply as A
from . import operator as O
from . import product as P
from . import tree as T


def nucleus(L, u0):
    return P.Potential(charges=[-1.0 / L], positions=[u0])


def kalos_step(phi, k, L, u0, mu, eps, max_level, op=None):
    """One pass of Steps 2-5.  Returns (phi_next, mu_next, E_new, norm_new)
    with norm_new the physical L2 norm of phi_new before normalisation."""
    V = nucleus(L, u0)
    Vphi = P.multiply(phi, k, V)                                          # Step 2
    if op is None:
        op = O.Operator(mu * L, 1.0, eps, k, max_level)
    g = A.apply_full(op, Vphi)                                            # Step 3
    phi_new = P.scale(g, -2.0 * L * L)
    nn = P.dot(phi_new, phi_new)                                          # Step 4
    e_num = (-P.dot(Vphi, phi_new) - 0.5 * mu * mu * nn
             + P.dot(P.multiply(phi_new, k, V), phi_new))
    E_new = e_num / nn
    norm_new = math.sqrt(nn * L ** 3)
    phi_next = P.scale(phi_new, 1.0 / norm_new)                           # Step 5
    mu_next = math.sqrt(-2.0 * E_new) if E_new < 0 else mu
    return phi_next, mu_next, E_new, norm_new


def slater_tree(k, L, u0, zeta, eps, max_level, init_level, terms):
    """A starting tree: Algorithm 1 on the Gaussian expansion ``terms`` =
    (c, a) of e^{-zeta r} (physical units), mapped to the unit cube."""
    c, a = terms
    dens = T.Density(c, a * L * L, [u0] * len(c))
    tree, _ = T.build_tree(dens, k, eps, max_level, init_level=init_level)
    return tree
