"""GB300-native leading-order matrix elements (per-event |M|^2 summed over
helicities and colours) behind a C ABI; see include/mg.h."""
