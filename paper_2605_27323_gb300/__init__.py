"""GB300-native Monte Carlo path tracer: megakernel and wavefront estimators behind a C ABI."""
