"""GB300-native encrypted GCN layer (placeholder; binding added below)."""
