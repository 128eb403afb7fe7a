"""GB300-native Newton power-flow hot path (arXiv 1711.10579, ExaGridPF)."""
