"""Galaxy light-profile mixture tables (model constants, passed as input data).

Each profile is a unit-flux circular Gaussian mixture sum_j nu_j N(0, tau_j I_2) whose
half-light radius is exactly 1; a galaxy component of variance tau_j is stretched by
the galaxy's scale/axis/angle covariance.  Written by `python -m synth.fit_mixtures`
(least-squares fit to the Sersic n=1 and n=4 laws, see that module).
"""
import numpy as np

# Exponential (Sersic n=1), 6 components.
EXP_NU = np.array([0.0006596951502967703, 0.008499948273535158, 0.056750668148803744, 0.22909140806738018, 0.4610677000650011, 0.24393058029498293])
EXP_TAU = np.array([0.0026964523198173673, 0.019832622513022816, 0.0868133713693027, 0.2965756227564619, 0.872162744212001, 2.3672623510096025])
# de Vaucouleurs (Sersic n=4), 8 components.
DEV_NU = np.array([0.00016023890226608196, 0.001477650972700837, 0.00773972860823985, 0.028967916143913062, 0.0835980906908277, 0.1889718131555343, 0.32221770578089337, 0.36686685574562483])
DEV_TAU = np.array([1.8377602381471976e-06, 3.154405920442516e-05, 0.00029861402151766113, 0.002189029452081167, 0.01433137495816934, 0.09284202670479808, 0.6780991051805976, 8.133158735894337])
