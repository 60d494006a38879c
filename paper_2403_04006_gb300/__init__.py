"""GB300-native permanents with repeated rows/columns (placeholder, binding follows)."""
