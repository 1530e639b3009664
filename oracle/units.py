"""Unit conversions of the paper (Sec. IV) -- TEST INFRASTRUCTURE ONLY.

With tau = 1 the lattice viscosity is nu = (2 tau - 1) / 6 = 1/6, and
matching the plasma viscosity nu' fixes dt = nu dx^2 / nu'.  rho_bar = 1 in
lattice units fixes dm = rho' dx^3.  A physical quantity converts to lattice
units by dividing by dx^a dt^b dm^c.
"""

NU_PLASMA = 1.09e-6      # m^2 / s (Sec. IV)
RHO_PLASMA = 1.03e3      # kg / m^3 (Sec. IV)
DX = 2.0 / 3.0 * 1e-6    # m (Sec. IV)


def lattice_viscosity(tau=1.0):
    return (2.0 * tau - 1.0) / 6.0


def dt(dx=DX, tau=1.0, nu_phys=NU_PLASMA):
    return lattice_viscosity(tau) * dx * dx / nu_phys


def dm(dx=DX, rho_phys=RHO_PLASMA):
    return rho_phys * dx ** 3


def energy_to_lattice(E, dx=DX):
    """J -> dm dx^2 / dt^2"""
    return E / (dm(dx) * dx * dx / dt(dx) ** 2)


def length_to_lattice(l, dx=DX):
    return l / dx


def rate_to_lattice(rate, dx=DX):
    """1/s -> 1/dt"""
    return rate * dt(dx)
