"""GB300-native EventTracer hot path: path tracing of 1 kHz frames and the
EvSNet spiking event generator, behind the C-ABI library ``libeventtracer``."""
