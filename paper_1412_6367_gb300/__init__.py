"""GB300-native azimuthal integration (Kieffer & Ashiotis, EuroSciPy 2014)."""
