"""GB300-native exponential drag solver for gas + N dust species (FP64, sm_103a)."""
