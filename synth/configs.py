"""The five benchmark workloads (lattice shapes, action parameters, seeds).

Parameters are bare, mass-normalised couplings in the tmLQCD input-file sense;
the operators use the hopping normalisation with 2*kappa*mu etc.  Seeds follow
one scheme: links 1000+c, right-hand sides 2000+c, batch problem i 3000+i,
preconditioner training configurations 4000+j, training pairs 5000+n.
"""
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple            # (X, Y, Z, T)
    kappa: float
    csw: float
    mu: float = 0.0        # light twisted mass
    mubar: float = 0.0     # heavy doublet: mu_sigma
    epsbar: float = 0.0    # heavy doublet: mu_delta
    bc_t: int = -1         # antiperiodic in time
    link_seed: int = 0
    rhs_seed: int = 0
    tol: float = 1e-10

    @property
    def volume(self):
        X, Y, Z, T = self.dims
        return X * Y * Z * T


LIGHT_4 = Workload("light 4^4 FP64 CG", (4, 4, 4, 4), 0.1394, 1.69, mu=0.01,
                   link_seed=1000, rhs_seed=2000, tol=1e-12)
LIGHT_32 = Workload("light 32^3x64 mixed-precision CG", (32, 32, 32, 64), 0.1400, 1.69,
                    mu=0.0015, link_seed=1001, rhs_seed=2001)
HEAVY_24 = Workload("heavy doublet 24^3x48 multishift CG", (24, 24, 24, 48), 0.1400, 1.69,
                    mubar=0.1246, epsbar=0.1350, link_seed=1002, rhs_seed=2002)
BATCH_DIMS = [(8, 8, 8, 16)] * 6 + [(12, 12, 12, 24)] * 6 + [(16, 16, 16, 32)] * 6 + \
    [(24, 24, 24, 48)] * 6
BATCH_MU = 0.002
PTC_48 = Workload("light 48^3x96 PTC-preconditioned FCG", (48, 48, 48, 96), 0.1394265, 1.69,
                  mu=0.00072, link_seed=1004, rhs_seed=2004)


def batch_workloads():
    return [Workload(f"batch member {i} {d}", d, 0.1400, 1.69, mu=BATCH_MU,
                     link_seed=3000 + i, rhs_seed=3100 + i) for i, d in enumerate(BATCH_DIMS)]


N_SHIFTS = 12


# two-level multigrid of the full operator at 48^3x96 (the PTC workload's action)
MG_PARAMS = dict(block=(4, 4, 4, 4), nvec=12, setup_steps=100, smooth_steps=8, coarse_tol=0.1,
                 coarse_maxiter=30, coarse_restart=16, restart=16, maxiter=1500)
