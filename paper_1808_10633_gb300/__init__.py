"""GB300-native WENO-Wombat MHD hot path (fifth-order characteristic WENO
sweeps, constrained transport, SSP-RK3, CFL) behind a small C ABI."""
