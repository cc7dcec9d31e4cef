"""GB300 thermal lattice Boltzmann (D3Q19 MRT + D3Q7 MRT) library and its binding."""
