"""GB300-native multi-function direct Monte Carlo integration (ZMCintegral-v5.1 method)."""
