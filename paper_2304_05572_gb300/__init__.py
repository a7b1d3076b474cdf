"""GB300-native (sm_103a) FP64 hot path of the hybrid WENO-AO gas-kinetic scheme."""
