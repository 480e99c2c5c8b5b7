"""GB300-native D2Q9 multiphase lattice Boltzmann library (arXiv:2403.11167)."""
