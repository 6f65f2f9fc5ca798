"""GB300-native complex-valued K-means ISDF (arXiv 2208.07731)."""
