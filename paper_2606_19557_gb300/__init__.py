"""GB300-native NEP loss + parameter-gradient hot path (placeholder; binding added below)."""
