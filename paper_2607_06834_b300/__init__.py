"""B300-native log-posterior and gradient engine for standardized Fourier-coefficient
pulsar-timing-array HMC (hot path: batched logp + gradient over chains)."""
