"""GB300-native Wiener-filter MAP objective, L-BFGS solver and band powers."""
