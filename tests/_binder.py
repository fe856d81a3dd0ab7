"""Worker of the Binder-cumulant pin (tests/test_oracle_physics.py): one
oracle chain, returning its sums of |m|^2, |m|^4 and the sample count."""
import oracle
import workloads


def binder_sums(args):
    L, T, seed, n_eq, n_meas = args
    o = oracle.Lattice((L, L, L), J=1.0, T=T, seed=seed, ring_cap=1)
    o.set_spins(workloads.random_spins(L ** 3, seed))
    o.sweep(n_eq)
    o.sweep(n_meas, measure=True)
    s = o.stats()
    return L, T, s["ml2"], s["ml4"], s["n"]
