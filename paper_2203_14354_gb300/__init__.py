"""GB300-native Monte Carlo propagation of LXe scintillation photons through a
triangle-mesh detector (optical simulation of a DARWIN-like dual-phase TPC)."""
