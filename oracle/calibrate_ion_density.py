"""Print the ion-density scale A of the synthetic downbranch model.

A is chosen so that the median Sobolev depth (Eq. 12, dilute-lte
populations of Eq. 5) of shell 0 in the first iteration -- T_R = 1e4 K and
the geometric dilution factor of Sect. 2.8 -- is e^-2.  tau is linear in A,
so one evaluation at A = 1 fixes it.  Uses the oracle only; the printed value
is stored as ``ION_DENSITY_SCALE`` in the package's ``synth`` module.

    python -m oracle.calibrate_ion_density
"""
import numpy as np

import oracle
from paper_1401_5469_gb300 import synth


def main():
    spec = synth.downbranch_model(ion_density_scale=1.0)
    t_rad = np.full(spec.n_shells, 1.0e4)
    w = oracle.geometric_dilution(spec)
    tau = oracle.plasma_tau(spec, t_rad, w)
    print(repr(float(np.exp(-2.0) / np.median(tau[0]))))


if __name__ == "__main__":
    main()
