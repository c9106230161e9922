"""GB300-native hierarchical factorization and solve of lambda*I + K."""
